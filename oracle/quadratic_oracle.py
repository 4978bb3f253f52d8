"""FP64 oracle of the ideal quadratic test model (paper section 4.1).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

What it computes:

* The misfit Hessian H_d = A A^T + V_r Lambda_r V_r^T (eq. (toy-hess)), A the
  order-1/2 PsiDO with the rank-3 symbol (eq. (toy-symbol))
      s_A(x, xi) = w(x) P(|xi|) (0.1 + cos^2(arg xi + pi x / x_max)) / (0.1 + (z / z_max)^2)
                 = sum_k a_k(x) b_k(xi)   (compound-angle expansion),
  applied as A v = sum_k a_k F^-1 (b_k F v) on the DFT grid (eq. (lr-psido)).
* The objective with the window W and the Matern prior:
      Phi(m) = 1/2 (W m - m*)^T H_d (W m - m*) + 1/2 m^T R m,
  i.e. Phi_d(W m) with Phi_d(m) = 1/2 m^T H_d m - b^T m + 1/2 b^T m*, b = H_d m*;
  gradient W H_d (W m - m*) + R m, Hessian W H_d W + R.

Readings (the paper describes P, w and V_r only qualitatively; stated in the
design notes):
* P(rho) = (rho / rho_c)^(1/2) exp(-(rho / rho_c)^4), rho in rad/m, rho_c = pi / (2 h)
  by default (half the Nyquist wavenumber).
* w = W = the product of 1D tapers t(i) = sin^2(pi/2 (i + 1/2) / L) over the L
  cells next to each edge (1 elsewhere; the smaller ramp where the two overlap).
* z = iz h, x = ix h, z_max = nz h, x_max = nx h; arg xi = atan2(xi_z, xi_x).
* V_r: for p = 1 .. r/2 the plane waves e^{-z/l} cos(2 pi p x / x_max) and
  e^{-z/l} sin(2 pi p x / x_max), l = z_max / 8, each scaled to unit norm
  (they are orthogonal on the periodic grid); Lambda_r given by the caller.

Pins: tests/test_quadratic_oracle.py.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle import lowrank_oracle as LO
from oracle import pdo_oracle as DO
from oracle import spd_oracle as SO


def taper(n: int, L: int) -> np.ndarray:
    i = np.arange(n, dtype=np.float64)
    if L <= 0:
        return np.ones(n)
    left = np.where(i < L, np.sin(0.5 * np.pi * (i + 0.5) / L) ** 2, 1.0)
    return np.minimum(left, left[::-1])


def window(nz: int, nx: int, L: int) -> np.ndarray:
    return np.outer(taper(nz, L), taper(nx, L))


def p_half(rho, rho_c: float):
    """P(rho): ~ rho^(1/2) at low frequency, cut off beyond rho_c."""
    t = np.asarray(rho, dtype=np.float64) / rho_c
    return np.sqrt(t) * np.exp(-t ** 4)


def depth_factor(nz: int, nx: int) -> np.ndarray:
    z = np.arange(nz, dtype=np.float64) / nz
    return np.repeat((1.0 / (0.1 + z ** 2))[:, None], nx, axis=1)


def symbol_A(nz, nx, h, rho_c, L, iz, ix, xi_z, xi_x):
    """s_A at grid point (iz, ix) and frequency (xi_z, xi_x) written out from eq. (toy-symbol)."""
    w = taper(nz, L)[iz] * taper(nx, L)[ix]
    z_rel, x_rel = iz / nz, ix / nx
    ang = np.arctan2(xi_z, xi_x)
    return (w * p_half(np.hypot(xi_z, xi_x), rho_c) * (0.1 + np.cos(ang + np.pi * x_rel) ** 2)
            / (0.1 + z_rel ** 2))


def factors(nz: int, nx: int, h: float, rho_c: float, L: int):
    """(a [3, nz, nx], b [3, nz, nx]) real: the rank-3 expansion, b in DFT order."""
    w = window(nz, nx, L) * depth_factor(nz, nx)
    x_rel = (np.arange(nx, dtype=np.float64) / nx)[None, :]
    a = np.stack([w, w * np.cos(2 * np.pi * x_rel), w * np.sin(2 * np.pi * x_rel)])
    XZ, XX = DO.grid_frequencies(nz, nx, h)
    P = p_half(np.hypot(XZ, XX), rho_c)
    ang = np.arctan2(XZ, XX)
    b = np.stack([0.6 * P, 0.5 * np.cos(2 * ang) * P, -0.5 * np.sin(2 * ang) * P])
    return a, b


def lowrank_modes(nz: int, nx: int, nlr: int) -> np.ndarray:
    if nlr % 2 or nlr < 0 or nlr // 2 >= nx // 2:
        raise ValueError("nlr must be even, with nlr / 2 below nx / 2")
    z = np.arange(nz, dtype=np.float64) / nz
    x = np.arange(nx, dtype=np.float64) / nx
    decay = np.exp(-8.0 * z)[:, None]
    V = []
    for p in range(1, nlr // 2 + 1):
        for f in (np.cos, np.sin):
            v = decay * f(2 * np.pi * p * x)[None, :]
            V.append(v / np.linalg.norm(v))
    return np.stack(V) if V else np.zeros((0, nz, nx))


@dataclass
class Quad:
    nz: int
    nx: int
    h: float
    rho_c: float
    L: int
    a: np.ndarray
    b: np.ndarray
    V: np.ndarray
    lam: np.ndarray
    W: np.ndarray


def make(nz: int, nx: int, h: float, lam, rho_c: float | None = None, L: int | None = None) -> Quad:
    rho_c = np.pi / (2 * h) if rho_c is None else rho_c
    L = max(1, min(nz, nx) // 8) if L is None else L
    lam = np.asarray(lam, dtype=np.float64)
    a, b = factors(nz, nx, h, rho_c, L)
    return Quad(nz, nx, h, rho_c, L, a, b, lowrank_modes(nz, nx, len(lam)), lam, window(nz, nx, L))


def apply_A(q: Quad, v):
    return DO.lr_apply(q.a, q.b, v)


def apply_AT(q: Quad, v):
    return SO.lr_apply_T(q.a, q.b, v)


def _each(f, v):
    v = np.asarray(v, dtype=np.float64)
    return np.stack([f(x) for x in v]) if v.ndim == 3 else f(v)


def apply_Hd_raw(q: Quad, v):
    """(A A^T + V Lambda V^T) v."""
    def one(x):
        c = q.V.reshape(len(q.lam), -1) @ x.ravel() * q.lam
        return apply_A(q, apply_AT(q, x)) + (c @ q.V.reshape(len(q.lam), -1)).reshape(x.shape)
    return _each(one, v)


def apply_Hd(q: Quad, v):
    """The misfit Hessian of Phi_d(W m): W (A A^T + V Lambda V^T) W v."""
    return _each(lambda x: q.W * apply_Hd_raw(q, q.W * x), v)


def objective(q: Quad, m, mstar, delta: float, gamma: float):
    """(Phi, gradient) of Phi(m) = Phi_d(W m) + 1/2 m^T R m."""
    m = np.asarray(m, dtype=np.float64)
    e = q.W * m - mstar
    He = apply_Hd_raw(q, e)
    Rm = LO.prior_R(m, q.h, delta, gamma)
    phi = 0.5 * np.vdot(e, He) + 0.5 * np.vdot(m, Rm)
    return float(phi), q.W * He + Rm


def objective_data_form(q: Quad, m, mstar, delta: float, gamma: float) -> float:
    """The same objective in the paper's form 1/2 u^T H_d u - b^T u + 1/2 b^T m*, u = W m, b = H_d m*."""
    u = q.W * np.asarray(m, dtype=np.float64)
    b = apply_Hd_raw(q, mstar)
    return float(0.5 * np.vdot(u, apply_Hd_raw(q, u)) - np.vdot(b, u) + 0.5 * np.vdot(b, mstar)
                 + 0.5 * np.vdot(m, LO.prior_R(m, q.h, delta, gamma)))
