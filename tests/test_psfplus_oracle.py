"""Pins of the FP64 PSF+ oracle (oracle/psfplus_oracle.py):

* the PSF symbol rows are the conjugated DFTs of the PSFs, and the PSF method
  in low-rank-symbol form (a_k = w_k, b_k = rows) agrees with the spatial row
  form of the PSF oracle away from the grid edges (the two forms of section 3.5);
* for PSFs p_k = f(x_k) K1 + K2 with f linear, the SVD basis and A0 = W U Sigma
  reproduce the rank-2 symbol f(x) K1^ + K2^ exactly inside the lattice;
* for a circulant operator (PSF rows all equal, PDO columns exact) PSF+ is exact;
* the refined A satisfies the normal equations of the regularised fit, and a
  wrong alpha does not.
"""
import numpy as np
import pytest

from oracle import pdo_oracle as DO
from oracle import psf_oracle as PO
from oracle import psfplus_oracle as PP

NZ, NX, H = 48, 64, 10.0
S, B = 8, 2                  # lattice 8 cells, R = 7
RHO0 = 0.15


def kernel(seed, rho=2):
    K = np.random.default_rng(seed).standard_normal((2 * rho + 1, 2 * rho + 1))
    return 0.5 * (K + K[::-1, ::-1])


def embed(K, R):
    """K (radius rho) in a (2R+1)^2 PSF window."""
    rho = (K.shape[0] - 1) // 2
    P = np.zeros((2 * R + 1, 2 * R + 1))
    P[R - rho:R + rho + 1, R - rho:R + rho + 1] = K
    return P


def test_rows_are_conjugated_dfts_and_match_the_spatial_row_form():
    R = PO.window_radius(S, B)
    C = PO.centers(NZ, NX, S)
    rng = np.random.default_rng(2)
    P = rng.standard_normal((len(C), 2 * R + 1, 2 * R + 1))
    rows = PP.psf_rows(P, NZ, NX)
    z, x = np.meshgrid(np.arange(NZ), np.arange(NX), indexing="ij")
    XZ, XX = DO.grid_frequencies(NZ, NX, H)
    k = 3
    direct = np.zeros((NZ, NX), dtype=complex)      # sum_d p(d) exp(i xi . d), written out
    for dz in range(-R, R + 1):
        for dx in range(-R, R + 1):
            direct += P[k, dz + R, dx + R] * np.exp(1j * (XZ * dz * H + XX * dx * H))
    np.testing.assert_allclose(rows[k], direct, atol=1e-10)
    # PSF method as a low-rank symbol (periodic) = spatial row form, away from the edges
    W = PO.weights(NZ, NX, S)
    v = rng.standard_normal((NZ, NX))
    v[:R + 1] = v[-R - 1:] = 0.0
    v[:, :R + 1] = v[:, -R - 1:] = 0.0
    got = DO.lr_apply(W, rows, v)
    want = PO.apply(P, v, S, B)
    np.testing.assert_allclose(got, want, atol=1e-11 * np.abs(want).max())


def test_rank_two_symbol_reproduced_by_svd_basis():
    R = PO.window_radius(S, B)
    C = PO.centers(NZ, NX, S)
    f = lambda z, x: 2.0 + 0.05 * z - 0.03 * x
    K1, K2 = embed(kernel(3), R), embed(kernel(4), R)
    P = np.stack([f(z, x) * K1 + K2 for z, x in C])
    cols = np.zeros((8, NZ, NX), dtype=complex)       # refinement not exercised here
    a, b, alpha, a0 = PP.psf_plus(P, S, B, cols, H, RHO0, 8)
    assert a0.shape[0] == 2
    s0 = np.einsum("izx,iab->zxab", a0, b)            # A0 B at every x, every xi
    rows1, rows2 = PP.psf_rows(K1[None], NZ, NX)[0], PP.psf_rows(K2[None], NZ, NX)[0]
    for (iz, ix) in [(4, 4), (20, 40), (44, 60), (11, 27)]:   # inside the lattice (points 4..44 x 4..60)
        want = f(iz, ix) * rows1 + rows2
        np.testing.assert_allclose(s0[iz, ix], want, atol=1e-10 * np.abs(want).max())


def test_exact_for_circulant_operator():
    K = kernel(7)
    rho = 2
    sig = np.conj(np.fft.fft2(np.pad(K, ((0, NZ - 5), (0, NX - 5)))))          # kernel at (0..4, 0..4)
    shift = np.exp(1j * 2 * np.pi * (rho * np.fft.fftfreq(NZ)[:, None] + rho * np.fft.fftfreq(NX)[None, :]))
    sig = sig * np.conj(shift)                                                   # centre it at the origin

    def circ(V):
        return np.stack([np.real(np.fft.ifft2(sig * np.fft.fft2(v))) for v in V])

    R = PO.window_radius(S, B)
    P = PO.build(circ, NZ, NX, S, B)
    for p in P:                                       # every PSF is the kernel
        np.testing.assert_allclose(p, embed(K, R), atol=1e-12)
    cols, _ = DO.build(circ, NZ, NX, H, RHO0, 8)
    a, b, alpha, a0 = PP.psf_plus(P, S, B, cols, H, RHO0, 8)
    assert a.shape[0] == 1
    v = np.random.default_rng(9).standard_normal((NZ, NX))
    want = circ(v[None])[0]
    np.testing.assert_allclose(DO.lr_apply(a, b, v), want, atol=1e-11 * np.abs(want).max())


def test_refinement_solves_the_regularised_fit():
    R = PO.window_radius(S, B)
    C = PO.centers(NZ, NX, S)
    rng = np.random.default_rng(5)
    P = np.stack([(1 + 0.1 * rng.standard_normal()) * embed(kernel(11), R) + 0.05 * rng.standard_normal(
        (2 * R + 1, 2 * R + 1)) for _ in C])
    cols = rng.standard_normal((8, NZ, NX)) + 1j * rng.standard_normal((8, NZ, NX))
    a, b, alpha, a0 = PP.psf_plus(P, S, B, cols, H, RHO0, 8)
    rr = a.shape[0]
    assert 1 < rr <= PP.MAX_RANK
    N = NZ * NX
    A, A0, Bm = a.reshape(rr, N).T, a0.reshape(rr, N).T, b.reshape(rr, N)
    idx, _, _ = DO.samples(NZ, NX, H, RHO0, 8)
    Ic = (idx[:, 0] % NZ) * NX + (idx[:, 1] % NX)
    Bc, Sc = Bm[:, Ic], cols.reshape(8, N).T
    assert alpha == pytest.approx(np.linalg.norm(Bc) ** 2 / rr)             # B has orthonormal rows
    grad = (A @ Bc - Sc) @ Bc.conj().T + alpha * (A - A0)
    assert np.abs(grad).max() < 1e-10 * np.abs(Sc @ Bc.conj().T).max()
    wrong = (A @ Bc - Sc) @ Bc.conj().T + 2 * alpha * (A - A0)
    assert np.abs(wrong).max() > 1e-3 * np.abs(Sc @ Bc.conj().T).max()
