"""Shared test helpers: oracle problems built from the same seeded inputs as the GPU path."""
import numpy as np

from oracle import oracle as O
from paper_2507_10804_gb300 import synth


def rel(a, b) -> float:
    """Relative L2 difference ||a - b|| / ||b|| (complex arrays keep their imaginary parts)."""
    dt = np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64
    a = np.asarray(a, dtype=dt).ravel()
    b = np.asarray(b, dtype=dt).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def f32(a) -> np.ndarray:
    """The float32 values the GPU receives, widened back to float64 for the oracle."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_problem(w: synth.Workload) -> O.Problem:
    return O.Problem(nz=w.nz, nx=w.nx, nb=w.nb, h=w.h, nt=w.nt, dt=w.dt, f0=w.f0, t0=w.t0, vmax=w.vmax,
                     src_iz=w.acq.src_iz, src_ix=w.acq.src_ix, rec_iz=w.acq.rec_iz, rec_ix=w.acq.rec_ix,
                     R=w.R, sigma=w.sigma)


def ragged_workload(nz=37, nx=71, nb=6, nt=150, ns=3, nr=7, k=3, seed=5, h=10.0, f0=20.0, sigma=0.8):
    """A small problem whose padded grid spans several tiles with ragged tails in both axes."""
    m = synth.gradient_grf_model(seed, nz, nx, h, 1500.0, 2400.0, std=80.0, corr_len=40.0)
    vmax = float(m.max())
    acq = synth.surface_acquisition(nx, ns, nr, src_iz=2, rec_iz=1)
    v = synth.smoothed_normal_vectors(seed + 1, k, nz, nx, 1.5)
    return synth.Workload(name="ragged", nz=nz, nx=nx, nb=nb, h=h, nt=nt, dt=synth.cfl_dt(h, vmax, 0.5), f0=f0,
                          t0=1.5 / f0, vmax=vmax, acq=acq, m=m, v=v, sigma=sigma)
