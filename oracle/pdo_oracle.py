"""FP64 oracle of the pseudo-differential-operator probing (PDO) approximation
and of the low-rank-symbol PsiDO apply it produces.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

What it computes (paper section 3.3, eq. (lr-psido); section 3.4; appendix A):

* A low-rank symbol s(x, xi) ~ sum_k a_k(x) b_k(xi) is applied as
      H~ v = sum_k D_{a_k} F^-1 D_{b_k} F v.
* PDO: the Hessian applied to a sum of r sinusoids at frequencies xi_k on a
  circle of radius rho0 (angles 2 pi k / r; pairs xi, -xi make the probe real)
  returns sum_k phi_k s(., xi_k); the symbol columns are separated in the
  frequency domain (each is clustered around its xi_k), demodulated, and
  interpolated with b_k(xi) = (rho / rho_k) w_k^circle(theta): linear in the
  magnitude, trigonometric (Fourier) interpolation over the angle.

Discrete readings (stated in the design notes):
* Grid frequencies are those of the DFT on the nz x nx interior grid with
  spacing h, in rad/m: xi = 2 pi (i / (nz h), j / (nx h)) with signed indices.
  A frequency xi = (xi_x, xi_z) = rho (cos theta, sin theta).
* Each sample xi_k = rho0 (cos theta_k, sin theta_k) is snapped to the nearest
  grid frequency (signed indices rounded half to even, so -xi_k snaps to minus
  the snapped xi_k); rho_k is the snapped radius, theta_k the nominal angle.
* Separation window of sample k: grid frequencies with |xi - xi_k| < rho0 sin(pi / r)
  (half the distance between neighbouring samples); rho0 + that radius must stay
  below the Nyquist frequency on both axes.
* w_k^circle(theta) = (1/r) [1 + 2 sum_{m=1}^{r/2-1} cos(m (theta - theta_k)) + cos(r/2 (theta - theta_k))].
* F is the unnormalised 2D DFT, F^-1 its inverse with the 1/N factor, so a grid
  Fourier mode phi_xi is mapped to s~(x, xi) phi_xi.

Pins: tests/test_pdo_oracle.py (exactness for a circulant order-1 symbol of
angular degree <= r/2 - 1, exact extraction of x-dependent columns of a
band-limited amplitude times a circulant operator, interpolation identities).
"""
from __future__ import annotations

import numpy as np


def grid_frequencies(nz: int, nx: int, h: float):
    """(xi_z [nz, nx], xi_x [nz, nx]) in rad/m, DFT order."""
    fz = 2.0 * np.pi * np.fft.fftfreq(nz, d=h)
    fx = 2.0 * np.pi * np.fft.fftfreq(nx, d=h)
    return np.meshgrid(fz, fx, indexing="ij")


def samples(nz: int, nx: int, h: float, rho0: float, r: int):
    """Snapped sample frequencies: signed DFT indices [r, 2] (iz, ix), radii rho_k [r], nominal angles [r]."""
    if r < 2 or r % 2:
        raise ValueError("r must be even and >= 2")
    theta = 2.0 * np.pi * np.arange(r) / r
    dz, dx = 2.0 * np.pi / (nz * h), 2.0 * np.pi / (nx * h)
    iz = np.round(rho0 * np.sin(theta) / dz).astype(np.int64)
    ix = np.round(rho0 * np.cos(theta) / dx).astype(np.int64)
    rho = np.hypot(iz * dz, ix * dx)
    return np.stack([iz, ix], axis=1), rho, theta


def window_radius(rho0: float, r: int) -> float:
    return rho0 * np.sin(np.pi / r)


def probe(nz: int, nx: int, h: float, rho0: float, r: int) -> np.ndarray:
    """v_p = sum_k exp(i x . xi_k) over the snapped samples (real: the samples come in +- pairs)."""
    idx, _, _ = samples(nz, nx, h, rho0, r)
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    v = np.zeros((nz, nx), dtype=np.complex128)
    for iz, ix in idx:
        v += np.exp(2j * np.pi * (iz * z / nz + ix * x / nx))
    assert np.abs(v.imag).max() < 1e-9 * max(1.0, np.abs(v.real).max())
    return v.real


def extract_columns(Hvp: np.ndarray, h: float, rho0: float, r: int) -> np.ndarray:
    """Symbol columns a_k(x) = s(x, xi_k), [r, nz, nx] complex, from the Hessian applied to the probe."""
    nz, nx = Hvp.shape
    idx, _, _ = samples(nz, nx, h, rho0, r)
    XZ, XX = grid_frequencies(nz, nx, h)
    U = np.fft.fft2(Hvp)
    rad = window_radius(rho0, r)
    nyq = np.pi / h
    if rho0 + rad >= nyq:
        raise ValueError("sample circle plus window reaches the Nyquist frequency")
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    cols = np.empty((r, nz, nx), dtype=np.complex128)
    for k, (iz, ix) in enumerate(idx):
        kz, kx = 2.0 * np.pi * iz / (nz * h), 2.0 * np.pi * ix / (nx * h)
        mask = np.hypot(XZ - kz, XX - kx) < rad
        part = np.fft.ifft2(U * mask)                         # phi_k s(., xi_k)
        cols[k] = part * np.exp(-2j * np.pi * (iz * z / nz + ix * x / nx))
    return cols


def circle_weights(theta: np.ndarray, r: int) -> np.ndarray:
    """[r, ...]: the trigonometric interpolation basis of r equally spaced angles, at angles theta."""
    tk = 2.0 * np.pi * np.arange(r) / r
    d = theta[None] - tk.reshape((r,) + (1,) * theta.ndim)
    w = np.ones_like(d)
    for m in range(1, r // 2):
        w += 2.0 * np.cos(m * d)
    w += np.cos((r // 2) * d)
    return w / r


def frequency_weights(nz: int, nx: int, h: float, rho0: float, r: int) -> np.ndarray:
    """b_k(xi) = (rho / rho_k) w_k^circle(theta), [r, nz, nx] real, on the DFT grid."""
    _, rho_k, _ = samples(nz, nx, h, rho0, r)
    XZ, XX = grid_frequencies(nz, nx, h)
    rho = np.hypot(XZ, XX)
    theta = np.arctan2(XZ, XX)
    return circle_weights(theta, r) * (rho[None] / rho_k[:, None, None])


def lr_apply(a: np.ndarray, b: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Re sum_k a_k F^-1 (b_k F v) for v [nz, nx] or [k, nz, nx] (eq. (lr-psido))."""
    v = np.asarray(v, dtype=np.float64)
    if v.ndim == 3:
        return np.stack([lr_apply(a, b, vj) for vj in v])
    V = np.fft.fft2(v)
    out = np.zeros(v.shape, dtype=np.complex128)
    for ak, bk in zip(a, b):
        out += ak * np.fft.ifft2(bk * V)
    return out.real


def build(hessian_apply, nz: int, nx: int, h: float, rho0: float, r: int = 8):
    """(a, b) of the PDO approximation of `hessian_apply` ([k, nz, nx] -> [k, nz, nx]) from one application."""
    Hvp = np.asarray(hessian_apply(probe(nz, nx, h, rho0, r)[None]), dtype=np.float64)[0]
    return extract_columns(Hvp, h, rho0, r), frequency_weights(nz, nx, h, rho0, r)
