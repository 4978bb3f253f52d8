"""Pins of the FP64 PSF-approximation oracle (oracle/psf_oracle.py) against what
the mathematics fixes, independent of any wave solver:

* the interpolation weights are a partition of unity, equal 1 at their own
  sample point, and reproduce linear functions exactly inside the lattice;
* with H = identity every PSF is a unit spike and the approximation is exact;
* for the symmetric operator H(x, y) = (f(x) + f(y)) / 2 * K(y - x) with f
  linear and K symmetric, the row-interpolation (PsiDO) form of the PSF method
  is exact inside the lattice (sum_k w_k(x) f(x_k) = f(x)), so a wrong weight,
  a mirrored offset (convolution instead of correlation), a transposed lattice
  index or a shifted window makes the comparison fail.
"""
import numpy as np
import pytest

from oracle import psf_oracle as PO

pytestmark = pytest.mark.filterwarnings("ignore")


def test_lattice_and_batches():
    cz0, cx0, na, nb = PO.lattice(36, 48, 6)
    assert (cz0, cx0, na, nb) == (3, 3, 6, 8)
    C = PO.centers(36, 48, 6)
    assert C.shape == (48, 2) and tuple(C[0]) == (3, 3) and tuple(C[-1]) == (33, 45)
    assert tuple(C[9]) == (9, 9)                     # point (a, b) = (1, 1) is k = a * nb + b
    V = PO.impulse_batches(36, 48, 6, 2)
    assert V.shape == (4, 36, 48) and V.sum() == 48
    for q in range(4):                               # points of one batch are 2 S apart
        z, x = np.nonzero(V[q])
        d = np.abs(z[:, None] - z[None, :]) + np.abs(x[:, None] - x[None, :])
        assert d[~np.eye(len(z), dtype=bool)].min() >= 12
    assert PO.window_radius(6, 2) == 5 and PO.window_radius(12, 2) == 11 and PO.window_radius(12, 1) == 5


@pytest.mark.parametrize("nz,nx,S", [(36, 48, 6), (17, 23, 5), (9, 40, 12), (5, 5, 8)])
def test_weights_partition_of_unity_and_linear_reproduction(nz, nx, S):
    W = PO.weights(nz, nx, S)
    C = PO.centers(nz, nx, S)
    assert W.min() >= 0.0
    np.testing.assert_allclose(W.sum(axis=0), 1.0, rtol=0, atol=1e-14)
    for k, (iz, ix) in enumerate(C):
        assert W[k, iz, ix] == pytest.approx(1.0, abs=1e-14)
    f = lambda z, x: 0.7 - 1.3 * z + 2.1 * x
    fk = np.array([f(z, x) for z, x in C])
    interp = np.einsum("k,kzx->zx", fk, W)
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    inside = (z >= C[:, 0].min()) & (z <= C[:, 0].max()) & (x >= C[:, 1].min()) & (x <= C[:, 1].max())
    np.testing.assert_allclose(interp[inside], f(z, x)[inside], rtol=0, atol=1e-12)
    # beyond the outermost points the weights are those of the nearest boundary (constant extrapolation)
    zc = np.clip(z, C[:, 0].min(), C[:, 0].max())
    xc = np.clip(x, C[:, 1].min(), C[:, 1].max())
    np.testing.assert_allclose(interp, f(zc, xc), rtol=0, atol=1e-12)


def test_identity_operator_is_reproduced():
    nz, nx, S, B = 20, 30, 6, 2
    P = PO.build(lambda v: v, nz, nx, S, B)
    R = PO.window_radius(S, B)
    spike = np.zeros((2 * R + 1, 2 * R + 1))
    spike[R, R] = 1.0
    for p in P:
        assert np.array_equal(p, spike)
    v = np.random.default_rng(1).standard_normal((nz, nx))
    np.testing.assert_allclose(PO.apply(P, v, S, B), v, rtol=0, atol=1e-14)


def _bilinear_amplitude_operator(nz, nx, rho, seed):
    """Dense H[x, y] = (f(x) + f(y)) / 2 * K(y - x), f linear, K symmetric with radius rho."""
    rng = np.random.default_rng(seed)
    K = rng.standard_normal((2 * rho + 1, 2 * rho + 1))
    K = 0.5 * (K + K[::-1, ::-1])                     # K(d) = K(-d)
    f = lambda z, x: 3.0 + 0.05 * z - 0.08 * x
    N = nz * nx
    H = np.zeros((N, N))
    for iz in range(nz):
        for ix in range(nx):
            for dz in range(-rho, rho + 1):
                for dx in range(-rho, rho + 1):
                    z, x = iz + dz, ix + dx
                    if 0 <= z < nz and 0 <= x < nx:
                        H[iz * nx + ix, z * nx + x] = 0.5 * (f(iz, ix) + f(z, x)) * K[dz + rho, dx + rho]
    assert np.array_equal(H, H.T)
    return H


@pytest.mark.parametrize("S,B,rho", [(6, 2, 2), (6, 1, 2), (6, 3, 2)])
def test_approximation_exact_for_linear_amplitude_translation_operator(S, B, rho):
    # grid chosen so the outermost sample points lie rho cells inside the edges: no PSF support is cut off
    nz, nx = 36, 48
    H = _bilinear_amplitude_operator(nz, nx, rho, seed=7)
    Happ = lambda V: (V.reshape(V.shape[0], -1) @ H.T).reshape(V.shape)
    P = PO.build(Happ, nz, nx, S, B)
    C = PO.centers(nz, nx, S)
    v = np.random.default_rng(3).standard_normal((2, nz, nx))
    got = PO.apply(P, v, S, B)
    want = Happ(v)
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    inside = (z >= C[:, 0].min()) & (z <= C[:, 0].max()) & (x >= C[:, 1].min()) & (x <= C[:, 1].max())
    for j in range(2):
        err = np.abs(got[j] - want[j])[inside].max() / np.abs(want[j]).max()
        assert err < 1e-13, err
        # outside the lattice the weights extrapolate f as a constant: not exact there
        assert np.abs(got[j] - want[j])[~inside].max() > 1e-6


def test_mirrored_offsets_are_detected():
    """A planted mistake -- convolution with p_k instead of correlation -- breaks the exactness pin."""
    nz, nx, S, B, rho = 36, 48, 6, 2, 2
    H = _bilinear_amplitude_operator(nz, nx, rho, seed=11)
    Happ = lambda V: (V.reshape(V.shape[0], -1) @ H.T).reshape(V.shape)
    P = PO.build(Happ, nz, nx, S, B)
    v = np.random.default_rng(5).standard_normal((nz, nx))
    want = Happ(v[None])[0]
    wrong = PO.apply(P[:, ::-1, ::-1].copy(), v, S, B)
    assert np.abs(wrong - want)[3:34, 3:46].max() / np.abs(want).max() > 1e-3
