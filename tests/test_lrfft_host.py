"""The four-step factorisation the fused low-rank-symbol transforms use (a DFT of
length L = R1 R2 as length-R2 DFTs over n2, the twiddles W_L^(n1 k2) and
length-R1 DFTs over n1, with n = n1 + R1 n2 and k = k2 + R2 k1), restated in
numpy for every length split of the kernels and checked against numpy's FFT,
forward and inverse, together with the radix-2 in-register DFT it is built
from.  Host only: the GPU tests check the kernels themselves."""
import numpy as np
import pytest

SPLITS = {16: (4, 4), 32: (8, 4), 64: (8, 8), 128: (16, 8), 256: (16, 16), 512: (32, 16)}


def bitrev(i, R):
    r, b = 0, 1
    while b < R:
        r = (r << 1) | (i & 1)
        i >>= 1
        b <<= 1
    return r


def dft_radix2(v, inv):
    """Radix-2 decimation in time after a bit-reversal permutation, twiddles exp(-+2 pi i p / (2 half))."""
    R = len(v)
    v = np.array([v[bitrev(i, R)] for i in range(R)], dtype=np.complex128)
    half = 1
    while half < R:
        for g in range(0, R, 2 * half):
            for p in range(half):
                w = np.exp((2j if inv else -2j) * np.pi * p / (2 * half))
                a, b = v[g + p], w * v[g + p + half]
                v[g + p], v[g + p + half] = a + b, a - b
        half *= 2
    return v


def four_step(x, R1, R2, inv):
    L = R1 * R2
    sgn = 1.0 if inv else -1.0
    Y = np.empty((R1, R2), dtype=np.complex128)
    for n1 in range(R1):                      # thread n1: length-R2 DFT over n2, then the twiddles
        v = dft_radix2([x[n1 + R1 * n2] for n2 in range(R2)], inv)
        Y[n1] = v * np.exp(sgn * 2j * np.pi * n1 * np.arange(R2) / L)
    X = np.empty(L, dtype=np.complex128)
    for k2 in range(R2):                      # thread k2: length-R1 DFT over n1
        u = dft_radix2(Y[:, k2], inv)
        X[k2 + R2 * np.arange(R1)] = u
    return X


@pytest.mark.parametrize("R", [2, 4, 8, 16, 32])
def test_radix2_register_dft(R):
    rng = np.random.default_rng(R)
    v = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    assert np.allclose(dft_radix2(v, False), np.fft.fft(v), rtol=0, atol=1e-12 * R)
    assert np.allclose(dft_radix2(v, True), np.fft.ifft(v) * R, rtol=0, atol=1e-12 * R)


@pytest.mark.parametrize("L", sorted(SPLITS))
def test_four_step_matches_fft(L):
    R1, R2 = SPLITS[L]
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    assert np.abs(four_step(x, R1, R2, False) - np.fft.fft(x)).max() < 1e-11 * L
    assert np.abs(four_step(x, R1, R2, True) - np.fft.ifft(x) * L).max() < 1e-11 * L


def test_2d_transform_is_columns_then_rows():
    """The 2D DFT of the applies as the kernels order it: column pass, then row pass."""
    rng = np.random.default_rng(7)
    nz, nx = 32, 16
    X = rng.standard_normal((nz, nx)) + 1j * rng.standard_normal((nz, nx))
    cols = np.stack([four_step(X[:, c], *SPLITS[nz], False) for c in range(nx)], axis=1)
    both = np.stack([four_step(cols[z], *SPLITS[nx], False) for z in range(nz)])
    assert np.abs(both - np.fft.fft2(X)).max() < 1e-10
