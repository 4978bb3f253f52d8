"""FP64 oracle of the SPD forms of the low-rank-symbol approximations (paper
section 3.7), of posterior sampling with them, and of the low-rank correction.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

What it computes:

* The transpose of the low-rank-symbol operator B v = Re sum_k a_k F^-1 (b_k F v)
  (eq. (lr-psido)) for real v, w:  B^T w = Re sum_k F^-1 (conj(b_k) F (conj(a_k) w)).
* Section 3.7: the square root of H_d is approximated instead of H_d, by the
  same procedure with a pointwise square root of the computed symbol rows or
  columns, negative values discarded: sqrt(max(Re s, 0)).  The approximation
  is then H~_d = B B^T, symmetric positive semi-definite.  For the PDO columns
  the radial extension follows the order of the operator approximated: the
  square root of an order-1 symbol is of order 1/2, so b_k(xi) =
  (|xi| / |xi_k|)^(1/2) w_k(theta) (for the order-1 H_d it is linear).
* Posterior samples with H~ = H~_d + R, R = A_pr^2 (section 2.2, Laplace
  approximation): with n1, n2 ~ N(0, I), y = A_pr n1 + B n2 ~ N(0, H~) and
  zeta = H~^-1 y ~ N(0, H~^-1); the solve is conjugate gradients to 1e-12.
* The low-rank correction (sections 3.1 and 3.7) of a base approximation
  H0 = H~_d + R of H = H_d + R: the leading eigenpairs of (H - H0) v = lambda H0 v,
  V^T H0 V = I, by the randomized double pass with the base in place of R:
      Y = H0^-1 (H_d - H~_d) Omega,  Q = H0-orthonormalised Y,
      T = Q^T (H_d - H~_d) Q = S Lambda S^T,  V = Q S[:, :r];
  then H~ = H0 + H0 V Lambda V^T H0, H~^-1 = H0^-1 - V D V^T (D = Lambda / (Lambda + 1)),
  and zeta = (I - V S_r V^T H0) z with z ~ N(0, H0^-1), S_r = I - (Lambda + I)^-1/2.
  With H~_d = 0 this is the low-rank approximation of section 3.1.

Pins: tests/test_spd_oracle.py.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, cg

from oracle import lowrank_oracle as LO
from oracle import pdo_oracle as DO


def lr_apply_T(a: np.ndarray, b: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Transpose of DO.lr_apply(a, b, .) for w [nz, nx] or [k, nz, nx]."""
    w = np.asarray(w, dtype=np.float64)
    if w.ndim == 3:
        return np.stack([lr_apply_T(a, b, x) for x in w])
    acc = np.zeros(w.shape, dtype=np.complex128)
    for ak, bk in zip(a, b):
        acc += np.conj(bk) * np.fft.fft2(np.conj(ak) * w)
    return np.fft.ifft2(acc).real


def sqrt_real(s: np.ndarray) -> np.ndarray:
    return np.sqrt(np.maximum(np.real(s), 0.0))


def pdo_sqrt(cols: np.ndarray, h: float, rho0: float, r: int):
    """(a, b) of the square-root PDO approximation from the PDO columns of H_d."""
    _, nz, nx = cols.shape
    _, rho_k, _ = DO.samples(nz, nx, h, rho0, r)
    XZ, XX = DO.grid_frequencies(nz, nx, h)
    rho = np.hypot(XZ, XX)
    b = DO.circle_weights(np.arctan2(XZ, XX), r) * np.sqrt(rho[None] / rho_k[:, None, None])
    return sqrt_real(cols), b


def spd_apply(a, b, v):
    """B B^T v."""
    return DO.lr_apply(a, b, lr_apply_T(a, b, v))


def _flat_op(f, shape):
    n = int(np.prod(shape))
    return LinearOperator((n, n), matvec=lambda x: f(x.reshape(shape)).ravel(), dtype=np.float64)


def solve(apply_op, rhs: np.ndarray, precond=None) -> np.ndarray:
    """apply_op^-1 rhs (SPD) by conjugate gradients to a relative residual of 1e-12."""
    shape = rhs.shape
    M = _flat_op(precond, shape) if precond is not None else None
    A = _flat_op(apply_op, shape)
    try:
        x, info = cg(A, rhs.ravel(), rtol=1e-12, atol=0.0, maxiter=20000, M=M)
    except TypeError:                       # scipy before 1.12 names the tolerance `tol`
        x, info = cg(A, rhs.ravel(), tol=1e-12, atol=0.0, maxiter=20000, M=M)
    if info != 0:
        raise RuntimeError("CG did not converge")
    return x.reshape(shape)


def posterior_sample(a, b, n1, n2, h, delta, gamma):
    """zeta = (B B^T + R)^-1 (A_pr n1 + B n2) for the square-root symbol (a, b)."""
    Hop = lambda x: spd_apply(a, b, x) + LO.prior_R(x, h, delta, gamma)
    y = LO.prior_A(np.asarray(n1, float), h, delta, gamma) + DO.lr_apply(a, b, n2)
    return solve(Hop, y, precond=lambda x: LO.prior_Rinv(x, h, delta, gamma))


def corrected_lowrank(resid_apply, base_apply, base_solve, omega: np.ndarray, rank: int):
    """(V [rank, ...], lam [rank]) of resid v = lambda base v, V^T base V = I, by the double pass."""
    k = omega.shape[0]
    shape = omega.shape[1:]
    Y = np.stack([base_solve(y) for y in np.asarray(resid_apply(omega), dtype=np.float64)]).reshape(k, -1)
    Q = Y
    for _ in range(2):
        BQ = np.stack([base_apply(q.reshape(shape)) for q in Q]).reshape(Q.shape[0], -1)
        G = Q @ BQ.T
        w, U = np.linalg.eigh(0.5 * (G + G.T))
        keep = w > 1e-12 * w.max()
        Q = (U[:, keep] / np.sqrt(w[keep])).T @ Q
    if rank > Q.shape[0]:
        raise ValueError("the test matrix spans fewer directions than the rank asked for")
    Z = np.asarray(resid_apply(Q.reshape((Q.shape[0],) + shape)), dtype=np.float64).reshape(Q.shape[0], -1)
    T = Q @ Z.T
    lam, S = np.linalg.eigh(0.5 * (T + T.T))
    order = np.argsort(lam)[::-1][:rank]
    return (S[:, order].T @ Q).reshape((rank,) + shape), lam[order]


def corrected_apply(base_apply, V, lam, v):
    """(H0 + H0 V Lambda V^T H0) v."""
    Vm = V.reshape(V.shape[0], -1)
    b0 = base_apply(v)
    c = (Vm @ b0.ravel()) * lam
    return b0 + base_apply((c @ Vm).reshape(v.shape))


def corrected_sample(base_apply, V, lam, z):
    """(I - V S_r V^T H0) z, S_r = I - (Lambda + I)^-1/2; z ~ N(0, H0^-1) gives N(0, H~^-1)."""
    Vm = V.reshape(V.shape[0], -1)
    s = 1.0 - 1.0 / np.sqrt(lam + 1.0)
    c = (Vm @ base_apply(z).ravel()) * s
    return z - (c @ Vm).reshape(z.shape)
