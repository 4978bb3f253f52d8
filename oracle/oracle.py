"""Python face of the FP64 CPU oracle (``hv_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this module, and this module
imports nothing from the product package.

Every routine here marshals numpy float64 arrays into the C oracle, which
writes out the plain definitions of the paper's operators:

* ``fwd_model``     -- the forward map f(m) of eq. (data): receiver samples of
                       the solution of eq. (pde).
* ``born``          -- F dm, F = grad f (the Born operator of eq. (grad)).
* ``adjoint``       -- F^T r, the migration operator F* of eq. (grad).
* ``misfit_grad``   -- Phi(m) = 1/2 ||f(m) - d||^2_{Gamma^-1} and its gradient,
                       eq. (grad) without the prior term.
* ``hessian_apply`` -- H_d v = F^T Gamma^{-1} F v, the matrix-free
                       Gauss-Newton Hessian action of section 3 ("two wave
                       equations per source", the forward field a third).
* ``hessian_image`` -- the same before the fold E^T: the sum over the
                       problem's sources of their extended images.
* ``wavefield``, ``solve_S``, ``solve_ST`` -- raw solves for the wavefield and
                       operator-level checks.

Parity status: every routine above is pinned by tests/test_oracle.py against
closed forms (2D Green's function, Laplacian exactness on polynomials),
adjoint identities, finite differences and a dense brute-force Hessian.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hv_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libhvoracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int), ("nx", ctypes.c_int), ("nb", ctypes.c_int),
        ("h", ctypes.c_double),
        ("nt", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("f0", ctypes.c_double), ("t0", ctypes.c_double),
        ("vmax", ctypes.c_double),
        ("R", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("ns", ctypes.c_int), ("nr", ctypes.c_int),
        ("src_iz", ctypes.POINTER(ctypes.c_int)), ("src_ix", ctypes.POINTER(ctypes.c_int)),
        ("rec_iz", ctypes.POINTER(ctypes.c_int)), ("rec_ix", ctypes.POINTER(ctypes.c_int)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        for name, args in {
            "or_ricker": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp],
            "or_sponge_q": [pp, dp],
            "or_extend": [pp, dp, dp],
            "or_fold": [pp, dp, dp],
            "or_laplacian": [pp, dp, dp],
            "or_fwd_model": [pp, dp, dp, ctypes.c_int],
            "or_wavefield": [pp, dp, ctypes.c_int, dp],
            "or_born": [pp, dp, ctypes.c_int, dp, dp, ctypes.c_int],
            "or_adjoint": [pp, dp, dp, dp, ctypes.c_int],
            "or_misfit_grad": [pp, dp, dp, dp, dp, ctypes.c_int],
            "or_hessian_apply": [pp, dp, ctypes.c_int, dp, dp, ctypes.c_int],
            "or_hessian_image": [pp, dp, ctypes.c_int, dp, dp, ctypes.c_int],
            "or_solve_S": [pp, dp, dp, dp],
            "or_solve_ST": [pp, dp, dp, dp],
        }.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int if name != "or_ricker" else None
    return _lib


@dataclass
class Problem:
    """Discrete problem: interior grid, sponge, time axis, source and receivers.

    Source and receiver positions are interior-grid (iz, ix) int32 nodes.
    ``vmax`` sizes the sponge damping rate and ``R`` is its target reflection
    coefficient; ``sigma`` is the noise standard deviation (Gamma = sigma^2 I).
    """
    nz: int
    nx: int
    nb: int
    h: float
    nt: int
    dt: float
    f0: float
    t0: float
    vmax: float
    src_iz: np.ndarray
    src_ix: np.ndarray
    rec_iz: np.ndarray  # [ns, nr]
    rec_ix: np.ndarray  # [ns, nr]
    R: float = 1e-3
    sigma: float = 1.0
    _keep: list = field(default_factory=list, repr=False)

    @property
    def ns(self) -> int:
        return int(np.asarray(self.src_iz).size)

    @property
    def nr(self) -> int:
        return int(np.asarray(self.rec_iz).shape[-1])

    @property
    def NZ(self) -> int:
        return self.nz + 2 * self.nb

    @property
    def NX(self) -> int:
        return self.nx + 2 * self.nb

    def _c(self) -> _Problem:
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))
                for a in (self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)]
        self._keep = arrs
        ip = ctypes.POINTER(ctypes.c_int)
        return _Problem(self.nz, self.nx, self.nb, self.h, self.nt, self.dt, self.f0, self.t0,
                        self.vmax, self.R, self.sigma, self.ns, self.nr,
                        *[a.ctypes.data_as(ip) for a in arrs])


def _d(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def ricker(nt: int, dt: float, f0: float, t0: float) -> np.ndarray:
    out = np.empty(nt)
    _load().or_ricker(nt, dt, f0, t0, _d(out))
    return out


def sponge_q(P: Problem) -> np.ndarray:
    """Sponge damping rate q [1/s] on the padded grid."""
    out = np.empty((P.NZ, P.NX))
    c = P._c()
    _load().or_sponge_q(ctypes.byref(c), _d(out))
    return out


def extend(P: Problem, m) -> np.ndarray:
    m = _f64(m)
    out = np.empty((P.NZ, P.NX))
    c = P._c()
    _load().or_extend(ctypes.byref(c), _d(m), _d(out))
    return out


def fold(P: Problem, gext) -> np.ndarray:
    gext = _f64(gext)
    out = np.empty((P.nz, P.nx))
    c = P._c()
    _load().or_fold(ctypes.byref(c), _d(gext), _d(out))
    return out


def laplacian(P: Problem, u) -> np.ndarray:
    u = _f64(u)
    out = np.empty((P.NZ, P.NX))
    c = P._c()
    _load().or_laplacian(ctypes.byref(c), _d(u), _d(out))
    return out


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed (out of host memory?)")


def fwd_model(P: Problem, m, nthreads=None) -> np.ndarray:
    """d[ns, nt, nr] = f(m)."""
    m = _f64(m)
    out = np.empty((P.ns, P.nt, P.nr))
    c = P._c()
    _check(_load().or_fwd_model(ctypes.byref(c), _d(m), _d(out), _threads(nthreads)), "fwd_model")
    return out


def wavefield(P: Problem, m, shot: int = 0) -> np.ndarray:
    """U[n] = u^{n+1} on the padded grid, shape [nt, NZ, NX]."""
    m = _f64(m)
    out = np.empty((P.nt, P.NZ, P.NX))
    c = P._c()
    _check(_load().or_wavefield(ctypes.byref(c), _d(m), int(shot), _d(out)), "wavefield")
    return out


def born(P: Problem, m, dm, nthreads=None) -> np.ndarray:
    """F dm for dm[k, nz, nx] (or [nz, nx]); returns [k, ns, nt, nr]."""
    m = _f64(m)
    dm = _f64(dm).reshape(-1, P.nz, P.nx)
    k = dm.shape[0]
    out = np.empty((k, P.ns, P.nt, P.nr))
    c = P._c()
    _check(_load().or_born(ctypes.byref(c), _d(m), k, _d(dm), _d(out), _threads(nthreads)), "born")
    return out


def adjoint(P: Problem, m, r, nthreads=None) -> np.ndarray:
    """F^T r for data r[ns, nt, nr]; returns [nz, nx]."""
    m = _f64(m)
    r = _f64(r).reshape(P.ns, P.nt, P.nr)
    out = np.empty((P.nz, P.nx))
    c = P._c()
    _check(_load().or_adjoint(ctypes.byref(c), _d(m), _d(r), _d(out), _threads(nthreads)), "adjoint")
    return out


def misfit_grad(P: Problem, m, dobs, nthreads=None):
    """(Phi, grad Phi) of the data misfit for observed data dobs[ns, nt, nr]."""
    m = _f64(m)
    dobs = _f64(dobs).reshape(P.ns, P.nt, P.nr)
    phi = np.zeros(1)
    g = np.empty((P.nz, P.nx))
    c = P._c()
    _check(_load().or_misfit_grad(ctypes.byref(c), _d(m), _d(dobs), _d(phi), _d(g),
                                  _threads(nthreads)), "misfit_grad")
    return float(phi[0]), g


def hessian_apply(P: Problem, m, v, nthreads=None) -> np.ndarray:
    """H_d v for v[k, nz, nx] (or [nz, nx]); returns the same leading shape."""
    m = _f64(m)
    v_in = _f64(v)
    v3 = v_in.reshape(-1, P.nz, P.nx)
    k = v3.shape[0]
    out = np.empty_like(v3)
    c = P._c()
    _check(_load().or_hessian_apply(ctypes.byref(c), _d(m), k, _d(v3), _d(out), _threads(nthreads)),
           "hessian_apply")
    return out.reshape(v_in.shape)


def hessian_image(P: Problem, m, v, nthreads=None) -> np.ndarray:
    """The extended image before the fold: [k, NZ, NX] with fold(P, ext[j]) == hessian_apply(P, m, v)[j]
    (the per-shot images of section 3 summed over the problem's shots in shot order)."""
    m = _f64(m)
    v3 = _f64(v).reshape(-1, P.nz, P.nx)
    k = v3.shape[0]
    out = np.empty((k, P.NZ, P.NX))
    c = P._c()
    _check(_load().or_hessian_image(ctypes.byref(c), _d(m), k, _d(v3), _d(out), _threads(nthreads)),
           "hessian_image")
    return out


def solve_S(P: Problem, m, F) -> np.ndarray:
    """U = S^{-1} F on the padded grid, F and U of shape [nt, NZ, NX]."""
    m = _f64(m)
    F = _f64(F)
    out = np.empty((P.nt, P.NZ, P.NX))
    c = P._c()
    _check(_load().or_solve_S(ctypes.byref(c), _d(m), _d(F), _d(out)), "solve_S")
    return out


def solve_ST(P: Problem, m, G) -> np.ndarray:
    """Lam = S^{-T} G on the padded grid, G and Lam of shape [nt, NZ, NX]."""
    m = _f64(m)
    G = _f64(G)
    out = np.empty((P.nt, P.NZ, P.NX))
    c = P._c()
    _check(_load().or_solve_ST(ctypes.byref(c), _d(m), _d(G), _d(out)), "solve_ST")
    return out
