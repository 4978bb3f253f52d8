"""FP64 oracle of the point-spread-function (PSF) Hessian approximation.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

What it computes (paper section 3.2, and section 3.5 "PSF method in PsiDO
formulation"):

* A PSF is the Hessian applied to a delta at a sample point x_k, read around
  x_k: p_k(d) = (H e_{x_k})[x_k + d].  Several PSFs come from one Hessian
  application to a sum of well-separated deltas.
* The approximation interpolates the symbol rows s(x_k, .) = (2 pi)^2 conj(p_k^)
  with weights w_k(x):  H v ~ (2 pi)^2 sum_k D_{w_k} F^-1 D_{conj(p_k^)} F v.
  On the grid, F^-1 D_{conj(p_k^)} F (with the paper's transform convention) is
  the correlation with p_k, so the operator is written out directly as

      (H~ v)(x) = sum_k w_k(x) sum_{|d|_inf <= R} p_k(d) v(x + d),   v = 0 off the grid.

Readings where the paper is silent (the same choices are stated in the design
notes; parity of the approximation's *quality* is not pinned, its arithmetic is):

* Sample points: a regular lattice of spacing S cells on the interior grid,
  first point at (floor(S/2), floor(S/2)), every point with iz < nz, ix < nx.
* Batches: B x B interleaved sub-lattices (point (a, b) in batch
  (a mod B) * B + (b mod B)); one Hessian application per batch, to the sum of
  unit impulses at its points (the paper's "4 H v for 36 PSFs" is 6 x 6 points
  with B = 2).
* Window: the box |d|_inf <= R with R = floor((B S - 1) / 2), so that the
  windows of points in one batch never overlap; PSF values whose x_k + d falls
  off the grid are zero.
* Weights: bilinear "hat" functions on the lattice (a partition of unity),
  constant beyond the outermost points.

Every function here is pinned in tests/test_psf_oracle.py: the weights against
the partition-of-unity and linear-reproduction identities, and the whole
build + apply against an operator for which the approximation is exact.
"""
from __future__ import annotations

import numpy as np


def lattice(nz: int, nx: int, S: int):
    """(cz0, cx0, na, nb): first sample point and the number of points along z and x."""
    if S < 1:
        raise ValueError("spacing must be >= 1")
    cz0, cx0 = S // 2, S // 2
    if cz0 >= nz or cx0 >= nx:
        raise ValueError("grid smaller than half a lattice spacing")
    na = (nz - 1 - cz0) // S + 1
    nb = (nx - 1 - cx0) // S + 1
    return cz0, cx0, na, nb


def window_radius(S: int, B: int) -> int:
    return (B * S - 1) // 2


def centers(nz: int, nx: int, S: int) -> np.ndarray:
    """[r, 2] int array of sample points (iz, ix), point k = a * nb + b."""
    cz0, cx0, na, nb = lattice(nz, nx, S)
    a, b = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
    return np.stack([cz0 + S * a.ravel(), cx0 + S * b.ravel()], axis=1)


def batch_of(nz: int, nx: int, S: int, B: int) -> np.ndarray:
    """Batch index of every sample point."""
    _, _, na, nb = lattice(nz, nx, S)
    a, b = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
    return ((a % B) * B + (b % B)).ravel()


def impulse_batches(nz: int, nx: int, S: int, B: int) -> np.ndarray:
    """[B*B, nz, nx]: the sum of unit impulses at each batch's sample points."""
    v = np.zeros((B * B, nz, nx))
    for (iz, ix), q in zip(centers(nz, nx, S), batch_of(nz, nx, S, B)):
        v[q, iz, ix] = 1.0
    return v


def extract(Hv: np.ndarray, S: int, B: int) -> np.ndarray:
    """PSFs [r, 2R+1, 2R+1] from the Hessian applied to the impulse batches [B*B, nz, nx]."""
    _, nz, nx = Hv.shape
    R = window_radius(S, B)
    C = centers(nz, nx, S)
    q = batch_of(nz, nx, S, B)
    P = np.zeros((len(C), 2 * R + 1, 2 * R + 1))
    for k, (iz, ix) in enumerate(C):
        for dz in range(-R, R + 1):
            for dx in range(-R, R + 1):
                z, x = iz + dz, ix + dx
                if 0 <= z < nz and 0 <= x < nx:
                    P[k, dz + R, dx + R] = Hv[q[k], z, x]
    return P


def _axis_weights(i: int, c0: int, S: int, n: int):
    """Lattice interval and bilinear weight along one axis: (a0, a1, f) with weights (1 - f, f)."""
    t = (i - c0) / S
    t = min(max(t, 0.0), n - 1.0)
    a0 = min(int(np.floor(t)), max(n - 2, 0))
    a1 = min(a0 + 1, n - 1)
    return a0, a1, t - a0


def weights(nz: int, nx: int, S: int) -> np.ndarray:
    """Dense [r, nz, nx] array of the interpolation weights w_k(x)."""
    cz0, cx0, na, nb = lattice(nz, nx, S)
    W = np.zeros((na * nb, nz, nx))
    for iz in range(nz):
        a0, a1, fz = _axis_weights(iz, cz0, S, na)
        for ix in range(nx):
            b0, b1, fx = _axis_weights(ix, cx0, S, nb)
            for a, wa in ((a0, 1.0 - fz), (a1, fz)):
                for b, wb in ((b0, 1.0 - fx), (b1, fx)):
                    W[a * nb + b, iz, ix] += wa * wb
    return W


def apply(P: np.ndarray, v: np.ndarray, S: int, B: int) -> np.ndarray:
    """(H~ v)(x) = sum_k w_k(x) sum_d p_k(d) v(x + d) for v[nz, nx] or [k, nz, nx]."""
    v = np.asarray(v, dtype=np.float64)
    if v.ndim == 3:
        return np.stack([apply(P, vj, S, B) for vj in v])
    nz, nx = v.shape
    R = window_radius(S, B)
    W = weights(nz, nx, S)
    vp = np.zeros((nz + 2 * R, nx + 2 * R))
    vp[R:R + nz, R:R + nx] = v
    out = np.zeros((nz, nx))
    for k in range(P.shape[0]):
        if not W[k].any():
            continue
        corr = np.zeros((nz, nx))          # sum_d p_k(d) v(x + d), every x
        for dz in range(2 * R + 1):
            for dx in range(2 * R + 1):
                if P[k, dz, dx] != 0.0:
                    corr += P[k, dz, dx] * vp[dz:dz + nz, dx:dx + nx]
        out += W[k] * corr
    return out


def build(hessian_apply, nz: int, nx: int, S: int, B: int) -> np.ndarray:
    """PSFs of the operator `hessian_apply` ([k, nz, nx] -> [k, nz, nx]) from B*B applications."""
    return extract(np.asarray(hessian_apply(impulse_batches(nz, nx, S, B)), dtype=np.float64), S, B)
