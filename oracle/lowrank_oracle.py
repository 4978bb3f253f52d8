"""FP64 oracle of the prior operator and the low-rank (LR) Hessian approximation.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

What it computes:

* The Matern prior (section 2.1): Gamma_pr = (delta I - gamma Lap_h)^{-2}, so the
  regularisation Hessian is R = A^2 with A = delta I - gamma Lap_h.  Lap_h is
  the 5-point Laplacian with homogeneous Neumann conditions (mirror ghost
  cells: u[-1] = u[0], u[n] = u[n-1]); the orthonormal DCT-II diagonalises it,
  -Lap_h cos-mode (k, l) = (4/h^2)(sin^2(pi k / 2 nz) + sin^2(pi l / 2 nx)) cos-mode.
* The LR approximation (section 3.1): the r leading eigenpairs of the
  generalised problem H_d v = lambda R v (V^T R V = I) by the randomized
  double-pass method with a given Gaussian test matrix Omega:
      Y = R^-1 H_d Omega,  Q = R-orthonormalised Y (through the eigen-decomposition of
      the R-Gram matrix, dropping directions below 1e-12 of the largest; twice),
      T = Q^T H_d Q,  T = S diag(lambda) S^T,  V = Q S[:, :r].
  Then H~_d + R = R + R V Lambda V^T R, (H~_d + R)^-1 = R^-1 - V D V^T with
  D = diag(lambda / (lambda + 1)), and zeta = (I - V S_r V^T R) z with z ~
  N(0, R^-1) (z = A^-1 n for n ~ N(0, I)), S_r = I - (Lambda + I)^{-1/2}, is a
  sample of N(0, (H~_d + R)^-1).

Pins: tests/test_lowrank_oracle.py.
"""
from __future__ import annotations

import numpy as np
from scipy.fft import dctn, idctn


def neumann_laplacian(v: np.ndarray, h: float) -> np.ndarray:
    """5-point Laplacian with mirror (homogeneous Neumann) ghost cells, written out."""
    p = np.pad(v, 1, mode="edge")
    return (p[2:, 1:-1] + p[:-2, 1:-1] + p[1:-1, 2:] + p[1:-1, :-2] - 4.0 * v) / h ** 2


def prior_A(v: np.ndarray, h: float, delta: float, gamma: float) -> np.ndarray:
    return delta * v - gamma * neumann_laplacian(v, h)


def prior_eigenvalues(nz: int, nx: int, h: float, delta: float, gamma: float) -> np.ndarray:
    kz = (4.0 / h ** 2) * np.sin(np.pi * np.arange(nz) / (2 * nz)) ** 2
    kx = (4.0 / h ** 2) * np.sin(np.pi * np.arange(nx) / (2 * nx)) ** 2
    return delta + gamma * (kz[:, None] + kx[None, :])


def prior_Ainv(v: np.ndarray, h: float, delta: float, gamma: float) -> np.ndarray:
    lam = prior_eigenvalues(v.shape[-2], v.shape[-1], h, delta, gamma)
    return idctn(dctn(v, type=2, norm="ortho", axes=(-2, -1)) / lam, type=2, norm="ortho", axes=(-2, -1))


def prior_R(v, h, delta, gamma):
    return prior_A(prior_A(v, h, delta, gamma), h, delta, gamma)


def prior_Rinv(v, h, delta, gamma):
    return prior_Ainv(prior_Ainv(v, h, delta, gamma), h, delta, gamma)


def _each(f, V, *args):
    return np.stack([f(v, *args) for v in V])


def r_orthonormalise(Y: np.ndarray, h, delta, gamma) -> np.ndarray:
    """Q [k', nz, nx] with Q^T R Q = I spanning Y [k, nz, nx]: the Gram matrix G = Y^T R Y = U W U^T
    gives Q = Y U W^-1/2 over the eigenvalues above 1e-12 of the largest (directions Y does not
    span are dropped); done twice."""
    Q = Y.reshape(Y.shape[0], -1)
    for _ in range(2):
        RQ = _each(prior_R, Q.reshape((Q.shape[0],) + Y.shape[1:]), h, delta, gamma).reshape(Q.shape[0], -1)
        G = Q @ RQ.T
        w, U = np.linalg.eigh(0.5 * (G + G.T))
        keep = w > 1e-12 * w.max()
        Q = (U[:, keep] / np.sqrt(w[keep])).T @ Q
    return Q.reshape((Q.shape[0],) + Y.shape[1:])


def lowrank(hessian_apply, omega: np.ndarray, rank: int, h, delta, gamma):
    """(V [rank, nz, nx], lam [rank]) of H_d v = lambda R v, double pass with test matrix omega [k, nz, nx]."""
    k = omega.shape[0]
    Y = _each(prior_Rinv, np.asarray(hessian_apply(omega), dtype=np.float64), h, delta, gamma)
    Q = r_orthonormalise(Y, h, delta, gamma)
    k = Q.shape[0]
    if rank > k:
        raise ValueError("the test matrix spans fewer directions than the rank asked for")
    Z = np.asarray(hessian_apply(Q), dtype=np.float64)
    T = Q.reshape(k, -1) @ Z.reshape(k, -1).T
    lam, S = np.linalg.eigh(0.5 * (T + T.T))
    order = np.argsort(lam)[::-1][:rank]
    V = (S[:, order].T @ Q.reshape(k, -1)).reshape((rank,) + omega.shape[1:])
    return V, lam[order]


def apply_H(V, lam, v, h, delta, gamma):
    """R V Lambda V^T R v for v [nz, nx] or [k, nz, nx]."""
    v = np.asarray(v, dtype=np.float64)
    if v.ndim == 3:
        return np.stack([apply_H(V, lam, x, h, delta, gamma) for x in v])
    Rv = prior_R(v, h, delta, gamma).ravel()
    c = V.reshape(V.shape[0], -1) @ Rv * lam
    return prior_R((c @ V.reshape(V.shape[0], -1)).reshape(v.shape), h, delta, gamma)


def apply_sample_factor(V, lam, v, h, delta, gamma):
    """(I - V S V^T R) A^-1 v, S = I - (Lambda + I)^-1/2: maps N(0, I) to N(0, (H~_d + R)^-1)."""
    v = np.asarray(v, dtype=np.float64)
    if v.ndim == 3:
        return np.stack([apply_sample_factor(V, lam, x, h, delta, gamma) for x in v])
    z = prior_Ainv(v, h, delta, gamma)
    Vm = V.reshape(V.shape[0], -1)
    s = 1.0 - 1.0 / np.sqrt(lam + 1.0)
    c = (Vm @ prior_R(z, h, delta, gamma).ravel()) * s
    return z - (c @ Vm).reshape(v.shape)
