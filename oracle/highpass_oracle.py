"""FP64 oracle of the high-pass filter applied to the Hessian before the PSF and
PDO approximations (paper section 3.2 and section 3.7: the low-frequency part
of H_d is removed before approximating, since it spoils the locality of the
point spread functions and the spectral separation of the probing).

TEST INFRASTRUCTURE ONLY: the test suite and the CPU-baseline leg of bench.py
call it; the product path never imports it, and it imports nothing from the
product package.

The paper does not specify the filter.  The reading taken here: a radial
Gaussian high-pass multiplier on the periodic 2D DFT of the nz x nx grid,

    (F_hp v)(x) = Re IDFT( phi(|xi|) DFT(v) ),   phi(rho) = 1 - exp(-rho^2 / (2 rho_c^2)),

with xi = (2 pi k_z / (nz h), 2 pi k_x / (nx h)) for the signed DFT indices
k_z, k_x, and the filtered Hessian F_hp H_d F_hp (the filter on both sides,
so the operator stays symmetric).  phi(0) = 0 (constants are removed) and
phi -> 1 above the cutoff rho_c [rad/m].

Parity status: pinned by tests/test_highpass_oracle.py (exact action on
cosine modes, symmetry and positive semi-definiteness of the dense filter).
"""
from __future__ import annotations

import numpy as np


def phi(rho, rho_c: float):
    """The radial multiplier 1 - exp(-rho^2 / (2 rho_c^2))."""
    rho = np.asarray(rho, dtype=np.float64)
    return 1.0 - np.exp(-(rho * rho) / (2.0 * rho_c * rho_c))


def wavenumbers(nz: int, nx: int, h: float):
    """|xi| [rad/m] at every DFT index (numpy's fft order), signed indices."""
    kz = np.fft.fftfreq(nz, d=1.0 / nz)          # signed integer indices
    kx = np.fft.fftfreq(nx, d=1.0 / nx)
    xz = 2.0 * np.pi * kz / (nz * h)
    xx = 2.0 * np.pi * kx / (nx * h)
    return np.sqrt(xz[:, None] ** 2 + xx[None, :] ** 2)


def highpass(v, h: float, rho_c: float) -> np.ndarray:
    """F_hp v for v[..., nz, nx]: the multiplier applied to the 2D DFT, real part of the inverse."""
    v = np.asarray(v, dtype=np.float64)
    nz, nx = v.shape[-2:]
    mult = phi(wavenumbers(nz, nx, h), rho_c)
    return np.real(np.fft.ifft2(np.fft.fft2(v, axes=(-2, -1)) * mult, axes=(-2, -1)))


def filtered_operator(apply, h: float, rho_c: float):
    """V -> F_hp apply(F_hp V) for V[k, nz, nx] (the operator the approximations are built from)."""
    def f(V):
        return highpass(apply(highpass(V, h, rho_c)), h, rho_c)
    return f
