"""Seeded synthetic inputs: velocity models, acquisition geometry and probe vectors.

This module generates INPUTS only.  It holds none of the wave-equation
arithmetic (no stencil, no source wavelet, no sponge, no imaging); both the
CUDA path and the CPU oracle receive the arrays it produces.  Every random
number comes from one counter-based generator, splitmix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), turned
into normals by the Box-Muller transform, so a seed fixes every byte.

The paper's Marmousi model (section 4.2) is not available; the models below
are seeded stand-ins with the paper's structure (a velocity increasing with
depth, layers, faults, a smooth background for the Gauss-Newton point), and
the acquisition mirrors its surface geometry: sources and receivers on the
top interior row, evenly spaced.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """The n outputs splitmix64(seed) produces at counters offset+1 .. offset+n."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def gaussian_smooth(field: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Periodic Gaussian smoothing by FFT (an input-recipe filter, not solver code)."""
    nz, nx = field.shape
    kz = np.fft.fftfreq(nz)[:, None]
    kx = np.fft.fftfreq(nx)[None, :]
    filt = np.exp(-2.0 * (np.pi * sigma_cells) ** 2 * (kz ** 2 + kx ** 2))
    return np.real(np.fft.ifft2(np.fft.fft2(field) * filt))


def grf(seed: int, nz: int, nx: int, h: float, std: float, corr_len: float) -> np.ndarray:
    """Zero-mean Gaussian random field with covariance ~ exp(-r^2 / (2 l^2)), rescaled to std exactly."""
    w = normal(seed, nz * nx).reshape(nz, nx)
    f = gaussian_smooth(w, corr_len / h / np.sqrt(2.0))
    f -= f.mean()
    sd = f.std()
    return f * (std / sd) if sd > 0 else f


@dataclass
class Acquisition:
    src_iz: np.ndarray   # [ns] int32, interior rows
    src_ix: np.ndarray   # [ns] int32, interior columns
    rec_iz: np.ndarray   # [ns, nr] int32
    rec_ix: np.ndarray   # [ns, nr] int32


def surface_acquisition(nx: int, ns: int, nr: int, src_iz: int = 0, rec_iz: int = 0) -> Acquisition:
    """Evenly spaced sources and receivers on one row, integer arithmetic only:
    ix_src(k) = floor((k + 1/2) nx / ns), ix_rec(r) = floor((r + 1/2) nx / nr)."""
    sx = np.array([((2 * k + 1) * nx) // (2 * ns) for k in range(ns)], dtype=np.int32)
    rx = np.array([((2 * r + 1) * nx) // (2 * nr) for r in range(nr)], dtype=np.int32)
    return Acquisition(
        src_iz=np.full(ns, src_iz, dtype=np.int32),
        src_ix=sx,
        rec_iz=np.full((ns, nr), rec_iz, dtype=np.int32),
        rec_ix=np.tile(rx, (ns, 1)).astype(np.int32),
    )


@dataclass
class Workload:
    """One seeded problem: grid, time axis, acquisition, model and vectors."""
    name: str
    nz: int
    nx: int
    nb: int
    h: float
    nt: int
    dt: float
    f0: float
    t0: float
    vmax: float
    acq: Acquisition
    m: np.ndarray          # [nz, nx] float64 velocity at the Gauss-Newton point
    v: np.ndarray          # [k, nz, nx] float64 vectors
    ckpt: int = 0          # snapshot budget per shot (0 = keep every step)
    sigma: float = 1.0
    R: float = 1e-3

    @property
    def ns(self) -> int:
        return int(self.acq.src_ix.size)

    @property
    def nr(self) -> int:
        return int(self.acq.rec_ix.shape[1])

    @property
    def k(self) -> int:
        return int(self.v.shape[0])


def cfl_dt(h: float, vmax: float, courant: float = 0.5) -> float:
    """dt such that vmax dt / h = courant."""
    return courant * h / vmax


def gradient_grf_model(seed: int, nz: int, nx: int, h: float, v_top=1500.0, v_bot=2500.0,
                       std=100.0, corr_len=100.0) -> np.ndarray:
    """Linear-in-depth velocity plus a Gaussian random field."""
    z = np.arange(nz, dtype=np.float64)[:, None] / max(nz - 1, 1)
    return v_top + (v_bot - v_top) * z + grf(seed, nz, nx, h, std, corr_len)


def layered_faulted_model(seed: int, nz: int, nx: int, h: float, n_layers=20, n_faults=3,
                          v_min=1500.0, v_max=5500.0, smooth_cells=10.0):
    """Layered model with normal faults, plus its smoothed copy (the GN point).

    Layer thicknesses and velocities (increasing v_min -> v_max with jitter) are
    seeded; each fault is a straight line with a seeded dip (50-70 degrees) and
    throw (50-200 m) whose hanging wall is shifted down.
    Returns (true_model, smooth_model).
    """
    u = uniform(seed, 4 * n_layers + 8 * n_faults + 8)
    cur = 0
    thick = 0.5 + u[cur:cur + n_layers]; cur += n_layers
    bounds = np.concatenate([[0.0], np.cumsum(thick) / np.sum(thick) * nz * h])
    jitter = (u[cur:cur + n_layers] - 0.5) * 0.6; cur += n_layers
    base = np.linspace(v_min, v_max, n_layers)
    step = (v_max - v_min) / max(n_layers - 1, 1)
    vel = np.clip(base + jitter * step, v_min, v_max)
    vel[0] = v_min
    zc = (np.arange(nz) + 0.5)[:, None] * h * np.ones((1, nx))
    xc = (np.arange(nx) + 0.5)[None, :] * h * np.ones((nz, 1))
    zeff = zc.copy()
    for f in range(n_faults):
        x0 = (0.15 + 0.7 * u[cur]) * nx * h
        dip = np.deg2rad(50.0 + 20.0 * u[cur + 1])
        throw = 50.0 + 150.0 * u[cur + 2]
        sgn = 1.0 if u[cur + 3] < 0.5 else -1.0
        cur += 8
        # signed horizontal distance from the fault plane x = x0 + sgn * z / tan(dip)
        dist = (xc - (x0 + sgn * zc / np.tan(dip))) * sgn
        zeff = np.where(dist > 0.0, zeff - throw, zeff)
    idx = np.clip(np.searchsorted(bounds, zeff, side="right") - 1, 0, n_layers - 1)
    true = vel[idx]
    true = np.clip(true, v_min, v_max)
    smooth = gaussian_smooth(np.pad(true, int(3 * smooth_cells), mode="edge"), smooth_cells)
    p = int(3 * smooth_cells)
    smooth = np.clip(smooth[p:p + nz, p:p + nx], v_min, v_max)
    return true, smooth


def smoothed_normal_vectors(seed: int, k: int, nz: int, nx: int, sigma_cells=2.0) -> np.ndarray:
    out = np.empty((k, nz, nx))
    for j in range(k):
        out[j] = gaussian_smooth(normal(seed + 7919 * j, nz * nx).reshape(nz, nx), sigma_cells)
    return out


def impulse_vectors(seed: int, k: int, nz: int, nx: int, spacing: int = 12) -> np.ndarray:
    """Sums of well-separated unit deltas on a lattice with a seeded offset per vector
    (the PSF construction inputs of section 3.2)."""
    out = np.zeros((k, nz, nx))
    u = uniform(seed, 2 * k)
    for j in range(k):
        oz = int(u[2 * j] * spacing)
        ox = int(u[2 * j + 1] * spacing)
        out[j, oz::spacing, ox::spacing] = 1.0
    return out


def rademacher_vectors(seed: int, k: int, nz: int, nx: int) -> np.ndarray:
    u = uniform(seed, k * nz * nx).reshape(k, nz, nx)
    return np.where(u < 0.5, -1.0, 1.0)


SEED_BASE = 20250714


def workload(cfg: int, *, nt: int | None = None, ns: int | None = None) -> Workload:
    """The seeded workloads.

    1: 64x64 at 10 m + 20-cell sponge, gradient + GRF model, one 15 Hz shot at
       (0, 32), 32 receivers every 2 cells, CFL 0.5, 600 steps, one smoothed
       N(0,1) vector.
    2: 384x1152 at 8 m + 40-cell sponge, layered/faulted 1500-5500 m/s (smooth
       GN point), 32 shots at 10 Hz, 384 receivers (24 m), 3000 steps,
       30 snapshots per shot, one smoothed N(0,1) vector.
    3: the model of 1, 32 shots, 600 steps, 64 vectors (48 impulse lattices
       with 12-cell spacing, 16 Rademacher).
    4: 256x256 at 10 m + 20-cell sponge, gradient + GRF model, 8 shots,
       1500 steps, 30 snapshots.
    ``nt``/``ns`` override the step and shot counts (smaller test cases).
    """
    seed = SEED_BASE + cfg
    if cfg in (1, 3):
        nz = nx = 64
        h, nb, f0 = 10.0, 20, 15.0
        m = gradient_grf_model(seed if cfg == 1 else SEED_BASE + 1, nz, nx, h)
        n_s = 1 if cfg == 1 else 32
        n_s = ns or n_s
        if cfg == 1 and n_s == 1:
            acq = Acquisition(np.array([0], np.int32), np.array([32], np.int32),
                              np.zeros((1, 32), np.int32),
                              np.tile(np.arange(1, 64, 2, dtype=np.int32), (1, 1)))
        else:
            acq = surface_acquisition(nx, n_s, 32)
        steps = nt or 600
        if cfg == 1:
            v = smoothed_normal_vectors(seed + 1, 1, nz, nx)
        else:
            v = np.concatenate([impulse_vectors(seed + 2, 48, nz, nx, 12),
                                rademacher_vectors(seed + 3, 16, nz, nx)])
        vmax = float(m.max())
        ckpt = 0
    elif cfg == 2:
        nz, nx, h, nb, f0 = 384, 1152, 8.0, 40, 10.0
        _, m = layered_faulted_model(seed, nz, nx, h)
        n_s = ns or 32
        acq = surface_acquisition(nx, n_s, 384)
        steps = nt or 3000
        v = smoothed_normal_vectors(seed + 1, 1, nz, nx)
        vmax = 5500.0
        ckpt = 30
    elif cfg == 4:
        nz = nx = 256
        h, nb, f0 = 10.0, 20, 15.0
        m = gradient_grf_model(seed, nz, nx, h)
        n_s = ns or 8
        acq = surface_acquisition(nx, n_s, 128)
        steps = nt or 1500
        v = smoothed_normal_vectors(seed + 1, 1, nz, nx)
        vmax = float(m.max())
        ckpt = 30
    else:
        raise ValueError(f"unknown workload {cfg}")
    dt = cfl_dt(h, vmax)
    return Workload(name=f"cfg{cfg}", nz=nz, nx=nx, nb=nb, h=h, nt=steps, dt=dt, f0=f0,
                    t0=1.5 / f0, vmax=vmax, acq=acq, m=m, v=v, ckpt=ckpt)


def perturbed_model(m: np.ndarray, h: float, seed: int, amp: float = 0.05, radius: float = 200.0) -> np.ndarray:
    """m times (1 + amp * Gaussian blob) at a seeded position (observed-data model)."""
    nz, nx = m.shape
    u = uniform(seed, 2)
    zc = (0.3 + 0.4 * u[0]) * nz * h
    xc = (0.3 + 0.4 * u[1]) * nx * h
    z = (np.arange(nz) + 0.5)[:, None] * h
    x = (np.arange(nx) + 0.5)[None, :] * h
    blob = np.exp(-((z - zc) ** 2 + (x - xc) ** 2) / (2.0 * radius ** 2))
    return m * (1.0 + amp * blob)
