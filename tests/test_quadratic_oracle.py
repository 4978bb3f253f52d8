"""Pins of the quadratic test model oracle (oracle/quadratic_oracle.py):

* the rank-3 factors a_k b_k sum to the symbol of eq. (toy-symbol) written out
  (the compound-angle expansion: a dropped term, a wrong sign or a swapped
  sine/cosine fails);
* A maps cos(xi . x) to s_A(x, xi) cos(xi . x) (b_k is even in xi), which fixes
  the DFT ordering, the axes and the angle convention of the apply;
* the transposed apply is the transpose of the dense matrix of A; H_d is
  symmetric positive semi-definite; the low-rank modes are orthonormal and
  decay with depth;
* the objective in residual form equals the paper's form with b = H_d m*, is
  1/2 m^T R m where W m = m*, and its gradient matches central differences
  (exact for a quadratic, up to rounding, at three step sizes).
"""
import numpy as np
import pytest

from oracle import lowrank_oracle as LO
from oracle import pdo_oracle as DO
from oracle import quadratic_oracle as QO

H = 10.0
LAM = [40.0, 30.0, 20.0, 12.0, 8.0, 5.0]


def test_rank3_expansion_is_the_symbol():
    nz, nx = 12, 20
    q = QO.make(nz, nx, H, LAM, L=2)
    XZ, XX = DO.grid_frequencies(nz, nx, H)
    s = np.einsum("kzx,kab->zxab", q.a, q.b)
    for iz in range(nz):
        for ix in range(nx):
            want = QO.symbol_A(nz, nx, H, q.rho_c, q.L, iz, ix, XZ, XX)
            np.testing.assert_allclose(s[iz, ix], want, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("fz,fx", [(1, 0), (0, 3), (2, 5), (-3, 4), (5, -2)])
def test_A_on_cosine_waves(fz, fx):
    nz, nx = 24, 32
    q = QO.make(nz, nx, H, LAM, L=3)
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    ph = 2 * np.pi * (fz * z / nz + fx * x / nx)
    xz, xx = 2 * np.pi * fz / (nz * H), 2 * np.pi * fx / (nx * H)
    got = QO.apply_A(q, np.cos(ph))
    want = QO.symbol_A(nz, nx, H, q.rho_c, q.L, z, x, xz, xx) * np.cos(ph)
    np.testing.assert_allclose(got, want, atol=1e-12 * np.abs(want).max())


def _dense(f, nz, nx):
    n = nz * nx
    return np.stack([f(e.reshape(nz, nx)).ravel() for e in np.eye(n)], axis=1)


def test_transpose_hessian_and_modes():
    nz, nx = 6, 10
    q = QO.make(nz, nx, H, LAM[:4], L=1)
    A = _dense(lambda v: QO.apply_A(q, v), nz, nx)
    AT = _dense(lambda v: QO.apply_AT(q, v), nz, nx)
    np.testing.assert_allclose(AT, A.T, atol=1e-13 * np.abs(A).max())
    Hd = _dense(lambda v: QO.apply_Hd(q, v), nz, nx)
    np.testing.assert_allclose(Hd, Hd.T, atol=1e-12 * np.abs(Hd).max())
    assert np.linalg.eigvalsh(Hd).min() > -1e-12 * np.abs(Hd).max()
    Wd = np.diag(q.W.ravel())
    np.testing.assert_allclose(Hd, Wd @ (A @ A.T + q.V.reshape(4, -1).T @ np.diag(q.lam) @ q.V.reshape(4, -1)) @ Wd,
                               atol=1e-12 * np.abs(Hd).max())
    Vm = q.V.reshape(4, -1)
    np.testing.assert_allclose(Vm @ Vm.T, np.eye(4), atol=1e-13)
    prof = np.abs(q.V[0]).max(axis=1)
    np.testing.assert_allclose(prof[1:] / prof[:-1], np.exp(-8.0 / nz), rtol=1e-12)


def test_window_and_taper():
    t = QO.taper(16, 4)
    np.testing.assert_allclose(t, t[::-1])
    assert t[4:12].min() == 1.0 and 0 < t[0] < t[1] < t[2] < t[3] < 1
    np.testing.assert_allclose(t[:4] + t[:4][::-1], 1.0, atol=1e-15)     # sin^2 + cos^2 ramp symmetry


def test_objective_forms_and_gradient():
    nz, nx = 10, 14
    q = QO.make(nz, nx, H, LAM, L=2)
    rng = np.random.default_rng(3)
    mstar, m, dm = rng.standard_normal((3, nz, nx))
    delta, gamma = 0.5, 30.0
    phi, g = QO.objective(q, m, mstar, delta, gamma)
    assert phi == pytest.approx(QO.objective_data_form(q, m, mstar, delta, gamma), rel=1e-12)
    m_at = mstar / q.W
    phi_at, _ = QO.objective(q, m_at, mstar, delta, gamma)
    assert phi_at == pytest.approx(0.5 * np.vdot(m_at, LO.prior_R(m_at, H, delta, gamma)), rel=1e-12)
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        fd = (QO.objective(q, m + eps * dm, mstar, delta, gamma)[0]
              - QO.objective(q, m - eps * dm, mstar, delta, gamma)[0]) / (2 * eps)
        errs.append(abs(fd - np.vdot(g, dm)))
    # the objective is quadratic: central differences are exact up to rounding
    assert max(errs) < 1e-9 * abs(np.vdot(g, dm))
