"""Pins of the prior operator and the low-rank (LR) approximation oracle
(oracle/lowrank_oracle.py):

* the Neumann Laplacian kills constants, is symmetric, and has the cosine modes
  as eigenvectors with the closed-form eigenvalues; A^-1 inverts A;
* for H_d = R W diag(mu) W^T R with W^T R W = I (rank 4), the randomized double
  pass recovers mu and the operator exactly;
* the sampling factor L satisfies L L^T = (R + R V Lambda V^T R)^-1 = R^-1 - V D V^T
  on a small grid (dense matrices), and a factor without the square root fails.
"""
import numpy as np
import pytest

from oracle import lowrank_oracle as LO

NZ, NX, H = 12, 16, 10.0
DELTA, GAMMA = 0.02, 40.0


def test_neumann_laplacian_and_prior_inverse():
    rng = np.random.default_rng(1)
    assert np.abs(LO.neumann_laplacian(np.full((NZ, NX), 3.7), H)).max() < 1e-14
    u, v = rng.standard_normal((2, NZ, NX))
    assert abs(np.vdot(u, LO.neumann_laplacian(v, H)) - np.vdot(LO.neumann_laplacian(u, H), v)) < 1e-12
    lam = LO.prior_eigenvalues(NZ, NX, H, DELTA, GAMMA)
    for k, l in [(0, 0), (1, 0), (3, 5), (11, 15)]:
        mode = np.cos(np.pi * k * (np.arange(NZ) + 0.5) / NZ)[:, None] * np.cos(np.pi * l * (np.arange(NX) + 0.5) / NX)[None, :]
        np.testing.assert_allclose(LO.prior_A(mode, H, DELTA, GAMMA), lam[k, l] * mode, atol=1e-12)
    np.testing.assert_allclose(LO.prior_A(LO.prior_Ainv(v, H, DELTA, GAMMA), H, DELTA, GAMMA), v, atol=1e-10)
    np.testing.assert_allclose(LO.prior_Rinv(LO.prior_R(v, H, DELTA, GAMMA), H, DELTA, GAMMA), v, atol=1e-9)


def _rank4_operator(seed):
    rng = np.random.default_rng(seed)
    W = LO.r_orthonormalise(rng.standard_normal((4, NZ, NX)), H, DELTA, GAMMA)
    mu = np.array([5.0, 3.0, 1.0, 0.5])

    def Hop(V):
        out = []
        for v in V:
            c = W.reshape(4, -1) @ LO.prior_R(v, H, DELTA, GAMMA).ravel() * mu
            out.append(LO.prior_R((c @ W.reshape(4, -1)).reshape(NZ, NX), H, DELTA, GAMMA))
        return np.stack(out)
    return Hop, mu


def test_double_pass_recovers_a_low_rank_operator():
    Hop, mu = _rank4_operator(3)
    omega = np.random.default_rng(4).standard_normal((8, NZ, NX))
    V, lam = LO.lowrank(Hop, omega, 4, H, DELTA, GAMMA)
    np.testing.assert_allclose(lam, mu, rtol=1e-9)
    Vm = V.reshape(4, -1)
    RV = np.stack([LO.prior_R(v, H, DELTA, GAMMA) for v in V]).reshape(4, -1)
    np.testing.assert_allclose(Vm @ RV.T, np.eye(4), atol=1e-9)
    x = np.random.default_rng(5).standard_normal((NZ, NX))
    want = Hop(x[None])[0]
    np.testing.assert_allclose(LO.apply_H(V, lam, x, H, DELTA, GAMMA), want, atol=1e-9 * np.abs(want).max())


def _dense(f, n):
    return np.stack([f(e.reshape(NZ, NX)).ravel() for e in np.eye(n)], axis=1)


def test_sampling_factor_and_inverse_identities():
    Hop, mu = _rank4_operator(6)
    V, lam = LO.lowrank(Hop, np.random.default_rng(7).standard_normal((7, NZ, NX)), 4, H, DELTA, GAMMA)
    N = NZ * NX
    Rm = _dense(lambda v: LO.prior_R(v, H, DELTA, GAMMA), N)
    Hm = _dense(lambda v: LO.apply_H(V, lam, v, H, DELTA, GAMMA), N)
    Lm = _dense(lambda v: LO.apply_sample_factor(V, lam, v, H, DELTA, GAMMA), N)
    C = np.linalg.inv(Rm + Hm)
    np.testing.assert_allclose(Lm @ Lm.T, C, atol=1e-8 * np.abs(C).max())
    Vm = V.reshape(4, -1).T
    np.testing.assert_allclose(np.linalg.inv(Rm) - Vm @ np.diag(lam / (lam + 1)) @ Vm.T, C, atol=1e-8 * np.abs(C).max())
    # planted mistake: S = I - (Lambda + I)^-1 instead of its square root
    z = _dense(lambda v: LO.prior_Ainv(v, H, DELTA, GAMMA), N)
    wrong = z - Vm @ np.diag(1 - 1 / (lam + 1)) @ Vm.T @ Rm @ z
    correction = np.abs(Vm @ np.diag(lam / (lam + 1)) @ Vm.T).max()
    assert np.abs(wrong @ wrong.T - C).max() > 0.05 * correction
