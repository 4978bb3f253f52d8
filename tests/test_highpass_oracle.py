"""Pins of the high-pass filter oracle (oracle/highpass_oracle.py) against what
the definition fixes: a Fourier multiplier acts on a cosine mode by scaling it
(a transposed axis, a wrong spacing or a missing 2 pi fails the scale), removes
constants, and is a symmetric positive semi-definite matrix with eigenvalues
phi(|xi|) in [0, 1)."""
import numpy as np

from oracle import highpass_oracle as HP


def test_cosine_modes_are_scaled_by_the_multiplier():
    nz, nx, h, rc = 24, 40, 8.0, 0.03
    z = np.arange(nz)[:, None] * h
    x = np.arange(nx)[None, :] * h
    for kz, kx in [(0, 1), (1, 0), (3, 5), (-2, 7), (12, 0), (5, 20), (7, -13)]:
        xi_z, xi_x = 2 * np.pi * kz / (nz * h), 2 * np.pi * kx / (nx * h)
        v = np.cos(xi_z * z + xi_x * x + 0.3)
        want = HP.phi(np.hypot(xi_z, xi_x), rc) * v
        assert np.abs(HP.highpass(v, h, rc) - want).max() < 1e-12


def test_constants_removed_and_multiplier_values():
    v = np.full((10, 12), 3.5)
    assert np.abs(HP.highpass(v, 5.0, 0.1)).max() < 1e-13
    assert HP.phi(0.0, 0.2) == 0.0
    assert abs(HP.phi(0.2, 0.2) - (1 - np.exp(-0.5))) < 1e-15
    assert HP.phi(10.0, 0.2) == 1.0


def test_dense_filter_symmetric_psd():
    nz, nx, h, rc = 6, 8, 10.0, 0.05
    E = np.eye(nz * nx).reshape(nz * nx, nz, nx)
    M = HP.highpass(E, h, rc).reshape(nz * nx, nz * nx)
    assert np.abs(M - M.T).max() < 1e-14
    w = np.linalg.eigvalsh(M)
    assert w.min() > -1e-14 and w.max() < 1.0
    # its eigenvalues are the multiplier on the DFT grid (each counted once)
    want = np.sort(HP.phi(HP.wavenumbers(nz, nx, h), rc).ravel())
    assert np.abs(np.sort(w) - want).max() < 1e-13


def test_filtered_operator_is_both_sided():
    nz, nx, h, rc = 8, 10, 10.0, 0.08
    rng = np.random.default_rng(3)
    A = rng.standard_normal((nz * nx, nz * nx))
    S = A @ A.T
    apply = lambda V: (S @ V.reshape(V.shape[0], -1).T).T.reshape(V.shape)
    f = HP.filtered_operator(apply, h, rc)
    E = np.eye(nz * nx).reshape(nz * nx, nz, nx)
    M = HP.highpass(E, h, rc).reshape(nz * nx, nz * nx)
    got = f(E).reshape(nz * nx, nz * nx).T
    assert np.abs(got - M @ S @ M).max() < 1e-10 * np.abs(S).max()
