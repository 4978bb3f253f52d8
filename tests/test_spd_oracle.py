"""Pins of the SPD / sampling / low-rank-correction oracle (oracle/spd_oracle.py):

* the transposed low-rank-symbol apply is the transpose of the dense matrix of
  the apply, for random complex factors;
* square-root PDO: for a circulant operator with symbol rho g(theta) whose
  square root rho^(1/2) g(theta)^(1/2) has angular degree below r/2, B B^T
  reproduces the operator exactly and B is the square-root operator; the
  linear radial extension (order 1) in its place fails; negative real parts
  are discarded;
* square-root PSF+: for a circulant operator with a non-negative symbol, B B^T
  reproduces it exactly;
* the sampler zeta = (B B^T + R)^-1 (A n1 + B n2) has covariance (B B^T + R)^-1
  (dense matrices on a small grid);
* the corrected low-rank double pass reduces to the section 3.1 routine for the
  base R, recovers an exact rank-4 correction of a general SPD base, and its
  sampling factor has covariance (H0 + H0 V Lambda V^T H0)^-1; without the
  square root it does not.
"""
import numpy as np
import pytest

from oracle import lowrank_oracle as LO
from oracle import pdo_oracle as DO
from oracle import psf_oracle as PO
from oracle import psfplus_oracle as PP
from oracle import spd_oracle as SO

H = 10.0


def _dense(f, nz, nx):
    return np.stack([f(e.reshape(nz, nx)).ravel() for e in np.eye(nz * nx)], axis=1)


def test_transpose_is_the_dense_transpose():
    nz, nx, r = 6, 10, 3
    rng = np.random.default_rng(1)
    a = rng.standard_normal((r, nz, nx)) + 1j * rng.standard_normal((r, nz, nx))
    b = rng.standard_normal((r, nz, nx)) + 1j * rng.standard_normal((r, nz, nx))
    M = _dense(lambda v: DO.lr_apply(a, b, v), nz, nx)
    MT = _dense(lambda v: SO.lr_apply_T(a, b, v), nz, nx)
    np.testing.assert_allclose(MT, M.T, atol=1e-13 * np.abs(M).max())
    S = _dense(lambda v: SO.spd_apply(a, b, v), nz, nx)
    np.testing.assert_allclose(S, M @ M.T, atol=1e-12 * np.abs(S).max())


NZ = NX = 64
RHO0 = 0.15


def _g_half(th):
    return 1.0 + 0.3 * np.cos(2 * th) + 0.2 * np.sin(2 * th)


def _circ(sym):
    XZ, XX = DO.grid_frequencies(NZ, NX, H)
    S = sym(np.hypot(XZ, XX), np.arctan2(XZ, XX))
    return lambda v: np.real(np.fft.ifft2(S * np.fft.fft2(v)))


def test_pdo_square_root_is_exact_for_a_circulant():
    Hop = _circ(lambda rho, th: rho * _g_half(th) ** 2)
    Bop = _circ(lambda rho, th: np.sqrt(rho) * _g_half(th))
    cols, _ = DO.build(lambda V: np.stack([Hop(x) for x in V]), NZ, NX, H, RHO0, 8)
    a, b = SO.pdo_sqrt(cols, H, RHO0, 8)
    # v without Nyquist content: there the grid has no -xi partner and the symbol's real part is
    # averaged with that of another frequency (the same happens to the circulant itself)
    V = np.fft.fft2(np.random.default_rng(2).standard_normal((NZ, NX)))
    V[NZ // 2, :] = 0
    V[:, NX // 2] = 0
    v = np.real(np.fft.ifft2(V))
    want_b, want_h = Bop(v), Hop(v)
    assert np.abs(DO.lr_apply(a, b, v) - want_b).max() < 1e-11 * np.abs(want_b).max()
    assert np.abs(SO.spd_apply(a, b, v) - want_h).max() < 1e-11 * np.abs(want_h).max()
    # planted mistake: the order-1 radial extension of the H_d approximation
    b1 = DO.frequency_weights(NZ, NX, H, RHO0, 8)
    assert np.abs(SO.spd_apply(a, b1, v) - want_h).max() > 0.05 * np.abs(want_h).max()


def test_negative_values_are_discarded():
    s = np.array([4.0 + 1.0j, -2.0 + 3.0j, 0.25 - 5.0j, -0.0])
    np.testing.assert_array_equal(SO.sqrt_real(s), [2.0, 0.0, 0.5, 0.0])


def test_psfplus_square_root_is_exact_for_a_circulant():
    S_, B_ = 8, 2
    kz, kx = np.zeros(NZ), np.zeros(NX)
    kz[[0, 1, -1]] = kx[[0, 1, -1]] = [0.5, 0.25, 0.25]
    K = np.outer(kz, kx)
    Khat = np.fft.fft2(K)                                      # cos^2 products: real and >= 0
    assert np.abs(Khat.imag).max() < 1e-14 and Khat.real.min() > -1e-14
    Hop = lambda v: np.real(np.fft.ifft2(Khat * np.fft.fft2(v)))
    Hb = lambda V: np.stack([Hop(x) for x in V])
    P = PO.build(Hb, NZ, NX, S_, B_)
    cols, _ = DO.build(Hb, NZ, NX, H, RHO0, 8)
    A, Bm, _, _ = PP.psf_plus(P, S_, B_, cols, H, RHO0, 8, spd=True)
    assert A.shape[0] == 1
    v = np.random.default_rng(5).standard_normal((NZ, NX))
    want = Hop(v)
    assert np.abs(SO.spd_apply(A, Bm, v) - want).max() < 1e-11 * np.abs(want).max()


def test_sampler_covariance():
    nz, nx = 6, 8
    n = nz * nx
    delta, gamma = 0.3, 20.0
    rng = np.random.default_rng(7)
    a = np.abs(rng.standard_normal((2, nz, nx))) + 0.1
    b = np.abs(rng.standard_normal((2, nz, nx)))
    cols = []
    for e in np.eye(2 * n):
        cols.append(SO.posterior_sample(a, b, e[:n].reshape(nz, nx), e[n:].reshape(nz, nx), H, delta, gamma).ravel())
    L = np.stack(cols, axis=1)
    Ht = _dense(lambda v: SO.spd_apply(a, b, v) + LO.prior_R(v, H, delta, gamma), nz, nx)
    C = np.linalg.inv(Ht)
    np.testing.assert_allclose(L @ L.T, C, atol=1e-9 * np.abs(C).max())


def test_corrected_lowrank_reduces_to_section_3_1_for_the_prior_base():
    nz, nx = 12, 16
    delta, gamma = 0.02, 40.0
    rng = np.random.default_rng(11)
    Wm = LO.r_orthonormalise(rng.standard_normal((4, nz, nx)), H, delta, gamma)
    mu = np.array([5.0, 3.0, 1.0, 0.5])

    def Hd(V):
        out = []
        for v in V:
            c = Wm.reshape(4, -1) @ LO.prior_R(v, H, delta, gamma).ravel() * mu
            out.append(LO.prior_R((c @ Wm.reshape(4, -1)).reshape(nz, nx), H, delta, gamma) + 1e-3 * v)
        return np.stack(out)
    omega = rng.standard_normal((7, nz, nx))
    V0, l0 = LO.lowrank(Hd, omega, 4, H, delta, gamma)
    V1, l1 = SO.corrected_lowrank(Hd, lambda v: LO.prior_R(v, H, delta, gamma),
                                  lambda v: LO.prior_Rinv(v, H, delta, gamma), omega, 4)
    np.testing.assert_allclose(l1, l0, rtol=1e-10)
    for i in range(4):
        s = np.sign(np.vdot(V0[i], V1[i]))
        np.testing.assert_allclose(s * V1[i], V0[i], atol=1e-8 * np.abs(V0[i]).max())


def test_corrected_lowrank_exact_recovery_and_covariance():
    nz, nx = 6, 8
    n = nz * nx
    rng = np.random.default_rng(13)
    G = rng.standard_normal((n, n))
    H0 = G @ G.T / n + np.eye(n)                     # a general SPD base
    C0 = np.linalg.cholesky(np.linalg.inv(H0))        # z = C0 n ~ N(0, H0^-1)
    Wr = rng.standard_normal((n, 4))
    Wr = Wr @ np.linalg.inv(np.linalg.cholesky(Wr.T @ H0 @ Wr).T)    # W^T H0 W = I
    mu = np.array([9.0, 4.0, 2.0, 0.7])
    Hres = H0 @ Wr @ np.diag(mu) @ Wr.T @ H0
    base = lambda v: (H0 @ v.ravel()).reshape(v.shape)
    resid = lambda V: np.stack([(Hres @ v.ravel()).reshape(nz, nx) for v in V])
    V, lam = SO.corrected_lowrank(resid, base, lambda v: np.linalg.solve(H0, v.ravel()).reshape(nz, nx),
                                  rng.standard_normal((6, nz, nx)), 4)
    np.testing.assert_allclose(lam, mu, rtol=1e-9)
    Vm = V.reshape(4, -1).T
    np.testing.assert_allclose(Vm.T @ H0 @ Vm, np.eye(4), atol=1e-9)
    Ht = H0 + Hres
    x = rng.standard_normal((nz, nx))
    np.testing.assert_allclose(SO.corrected_apply(base, V, lam, x).ravel(), Ht @ x.ravel(), rtol=1e-9, atol=1e-9)
    L = np.stack([SO.corrected_sample(base, V, lam, (C0 @ e).reshape(nz, nx)).ravel() for e in np.eye(n)], axis=1)
    C = np.linalg.inv(Ht)
    np.testing.assert_allclose(L @ L.T, C, atol=1e-9 * np.abs(C).max())
    # planted mistake: S = I - (Lambda + I)^-1
    s = 1 - 1 / (lam + 1)
    wrong = C0 - Vm @ np.diag(s) @ Vm.T @ H0 @ C0
    assert np.abs(wrong @ wrong.T - C).max() > 0.05 * np.abs(Vm @ np.diag(lam / (lam + 1)) @ Vm.T).max()
