"""Pins of the FP64 PDO / low-rank-symbol oracle (oracle/pdo_oracle.py) against
what the mathematics fixes:

* the angular weights are the trigonometric interpolation basis (Kronecker
  delta at the samples, partition of unity, exact on trigonometric
  polynomials of degree < r/2 and on cos(r/2 theta));
* for a circulant operator whose symbol is rho * g(theta) with g of degree
  <= 3, the probe-separate-interpolate construction reproduces the operator
  exactly on a grid with equal frequency spacing (snapping keeps the angles);
* for D_f C with a band-limited amplitude f, each extracted symbol column is
  f(x) sigma(xi_k) exactly and the approximation is exact -- a sign error in
  the demodulation, a wrong radius or a transposed axis fails one of them.
"""
import numpy as np
import pytest

from oracle import pdo_oracle as DO

NZ = NX = 64
H = 10.0
RHO0 = 0.15          # rad/m; Nyquist is pi / h = 0.314


def sigma(XZ, XX):
    """rho g(theta), g of angular degree 3; odd harmonics imaginary (a real operator has
    sigma(-xi) = conj(sigma(xi)))."""
    rho = np.hypot(XZ, XX)
    th = np.arctan2(XZ, XX)
    return rho * (1.0 + 0.4 * np.cos(2 * th) - 0.25 * np.sin(2 * th) + 0.1j * np.cos(3 * th))


def circulant(v):
    XZ, XX = DO.grid_frequencies(NZ, NX, H)
    return np.real(np.fft.ifft2(sigma(XZ, XX) * np.fft.fft2(v)))


def test_samples_and_probe():
    idx, rho, th = DO.samples(NZ, NX, H, RHO0, 8)
    assert idx.shape == (8, 2)
    assert np.array_equal(idx[:4], -idx[4:])                    # +- pairs
    d = 2 * np.pi / (NZ * H)
    np.testing.assert_allclose(np.arctan2(idx[:, 0] * d, idx[:, 1] * d) % (2 * np.pi), th, atol=1e-12)
    v = DO.probe(NZ, NX, H, RHO0, 8)
    spec = np.abs(np.fft.fft2(v))
    peaks = np.argwhere(spec > 1e-6 * spec.max())
    assert len(peaks) == 8                                        # exactly the 8 sample frequencies
    assert v[0, 0] == pytest.approx(8.0)


@pytest.mark.parametrize("r", [4, 8, 16])
def test_circle_weights_interpolate_trigonometric_polynomials(r):
    tk = 2 * np.pi * np.arange(r) / r
    W = DO.circle_weights(tk, r)
    np.testing.assert_allclose(W, np.eye(r), atol=1e-13)
    th = np.linspace(-3.0, 9.0, 101)
    W = DO.circle_weights(th, r)
    np.testing.assert_allclose(W.sum(axis=0), 1.0, atol=1e-13)
    for m in range(1, r // 2):
        for f in (np.cos, np.sin):
            np.testing.assert_allclose(f(m * tk) @ W, f(m * th), atol=1e-12)
    np.testing.assert_allclose(np.cos(r // 2 * tk) @ W, np.cos(r // 2 * th), atol=1e-12)


def test_exact_for_circulant_order_one_symbol():
    a, b = DO.build(lambda V: np.stack([circulant(x) for x in V]), NZ, NX, H, RHO0, 8)
    v = np.random.default_rng(4).standard_normal((2, NZ, NX))
    got = DO.lr_apply(a, b, v)
    for j in range(2):
        want = circulant(v[j])
        assert np.abs(got[j] - want).max() < 1e-11 * np.abs(want).max()
    # each column is the constant symbol value at its sample
    idx, _, _ = DO.samples(NZ, NX, H, RHO0, 8)
    d = 2 * np.pi / (NZ * H)
    for k, (iz, ix) in enumerate(idx):
        np.testing.assert_allclose(a[k], sigma(iz * d, ix * d), rtol=1e-12, atol=1e-14)


def test_columns_of_band_limited_amplitude_times_circulant_are_exact():
    z, x = np.meshgrid(np.arange(NZ), np.arange(NX), indexing="ij")
    f = 1.0 + 0.3 * np.cos(2 * np.pi * (2 * z / NZ + x / NX)) - 0.1 * np.sin(2 * np.pi * (z / NZ - 3 * x / NX))
    Hop = lambda v: f * circulant(v)
    a, b = DO.build(lambda V: np.stack([Hop(x_) for x_ in V]), NZ, NX, H, RHO0, 8)
    idx, _, _ = DO.samples(NZ, NX, H, RHO0, 8)
    d = 2 * np.pi / (NZ * H)
    for k, (iz, ix) in enumerate(idx):
        np.testing.assert_allclose(a[k], f * sigma(iz * d, ix * d), rtol=1e-11, atol=1e-13)
    v = np.random.default_rng(8).standard_normal((NZ, NX))
    want = Hop(v)
    assert np.abs(DO.lr_apply(a, b, v) - want).max() < 1e-11 * np.abs(want).max()
    # planted mistake: demodulating with +xi_k instead of -xi_k
    k = 1
    iz, ix = idx[k]
    wrong = a[k] * np.exp(4j * np.pi * (iz * z / NZ + ix * x / NX))
    assert np.abs(wrong - f * sigma(iz * d, ix * d)).max() > 0.1


def test_window_must_stay_below_nyquist():
    with pytest.raises(ValueError):
        DO.extract_columns(np.zeros((NZ, NX)), H, 0.3, 8)
