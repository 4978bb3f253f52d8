"""Python face of libhv: one ``Problem`` per grid + acquisition, calls that take
and return CUDA tensors.  Marshalling only -- every step of the path runs in
the library's kernels on the caller's current CUDA stream.

Names follow the C ABI (include/hv.h): fwd_model, wavefield, born, migrate,
misfit_grad, hessian_apply.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (HV_CKPT_ALL, HV_LAUNCH_DATAFLOW, HV_LAUNCH_PDL, HV_LAUNCH_PLAIN, HV_OP_BORN, HV_OP_FWD, HV_OP_GRAD,
                   HV_OP_HV, HV_OP_MIGRATE, HV_OP_WAVEFIELD, check)

__all__ = ["Problem", "HV_CKPT_ALL", "checkpoint_schedule"]


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def _dev(t: torch.Tensor, dtype, shape, name: str, device) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: expected contiguous {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
    if t.device != device:
        raise ValueError(f"{name} is on {t.device}, the problem on {device}")
    return t.data_ptr()


class Problem:
    """A discretised acquisition (grid, sponge, time axis, sources, receivers) on one GPU."""

    def __init__(self, nz, nx, nb, h, nt, dt, f0, t0, vmax, src_iz, src_ix, rec_iz, rec_ix,
                 R=1e-3, sigma=1.0, device=None):
        self.lib = _lib.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nz, self.nx, self.nb, self.h = int(nz), int(nx), int(nb), float(h)
        self.nt, self.dt = int(nt), float(dt)
        self.src_iz, self.src_ix = _i32(src_iz), _i32(src_ix)
        self.rec_iz, self.rec_ix = _i32(rec_iz), _i32(rec_ix)
        self.ns = self.src_iz.size
        self.nr = self.rec_iz.size // max(self.ns, 1)
        self.sigma = float(sigma)
        g = _lib.HvGrid(self.nz, self.nx, self.nb, self.h)
        a = _lib.HvAcq(self.ns, self.src_iz.ctypes.data_as(_lib.ip), self.src_ix.ctypes.data_as(_lib.ip),
                       self.nr, self.rec_iz.ctypes.data_as(_lib.ip), self.rec_ix.ctypes.data_as(_lib.ip),
                       self.nt, self.dt, float(f0), float(t0), float(vmax), float(R), self.sigma)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hv_create(ctypes.byref(g), ctypes.byref(a), ctypes.byref(handle)))
        self._h = handle
        self._ws = {}
        self.NZ, self.NX = self.nz + 2 * self.nb, self.nx + 2 * self.nb

    @classmethod
    def from_workload(cls, w, device=None) -> "Problem":
        return cls(w.nz, w.nx, w.nb, w.h, w.nt, w.dt, w.f0, w.t0, w.vmax, w.acq.src_iz, w.acq.src_ix,
                   w.acq.rec_iz, w.acq.rec_ix, R=w.R, sigma=w.sigma, device=device)

    def close(self):
        if getattr(self, "_h", None):
            self.lib.hv_destroy(self._h)
            self._h = None
            self._ws.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- profiling
    def profile(self, enable: bool = True) -> None:
        """Bracket every kernel launch of this problem with CUDA events (hv_profile)."""
        check(self.lib.hv_profile(self._h, int(bool(enable))))

    def profile_read(self) -> dict:
        """{kind: (launches, total_ms)} for kinds fwd, advance, adj, other; clears the record."""
        n = (ctypes.c_longlong * _lib.HV_K_COUNT)()
        t = (ctypes.c_double * _lib.HV_K_COUNT)()
        check(self.lib.hv_profile_read(self._h, n, t))
        names = ("fwd", "advance", "adj", "other")
        return {names[i]: (int(n[i]), float(t[i])) for i in range(_lib.HV_K_COUNT)}

    # ---------------------------------------------------------------- tiles, autotuning, graphs
    def tiles(self) -> tuple:
        """Tile configuration per kernel kind (forward+Born, forward-only, adjoint)."""
        c = (ctypes.c_int * 3)()
        check(self.lib.hv_get_tiles(self._h, c))
        return tuple(c)

    def set_tiles(self, cfg) -> None:
        c = (ctypes.c_int * 3)(*[int(x) for x in cfg])
        check(self.lib.hv_set_tiles(self._h, c))

    def set_graphs(self, enable: bool = True) -> None:
        """Replay the H v launch sequence as a CUDA graph (hv_set_graphs)."""
        check(self.lib.hv_set_graphs(self._h, int(bool(enable))))

    def status(self) -> int:
        """Device status of the handle's kernels since the last call (HV_OK or HV_ETIMEOUT); resets it."""
        c = ctypes.c_int()
        check(self.lib.hv_status(self._h, ctypes.byref(c)))
        return c.value

    def set_step_fusion(self, enable: bool = True) -> None:
        """Recompute two forward steps per launch where possible (hv_set_step_fusion)."""
        check(self.lib.hv_set_step_fusion(self._h, int(bool(enable))))

    def set_resident(self, enable: bool = True) -> bool:
        """Shared-memory-resident H v with every level stored (hv_set_resident); returns whether this
        problem's grid fits the resident kernels."""
        check(self.lib.hv_set_resident(self._h, int(bool(enable))))
        return bool(self.lib.hv_resident_fits(self._h))

    def set_launch_mode(self, mode: int) -> None:
        """How stencil steps follow one another: HV_LAUNCH_PLAIN, _PDL or _DATAFLOW (hv_set_launch_mode)."""
        check(self.lib.hv_set_launch_mode(self._h, int(mode)))

    def autotune(self, k: int = 1, cache: str | None = None) -> tuple:
        """Pick the fastest tile shape per kernel kind for k vectors (hv_autotune).

        The choice is cached in a JSON file (``cache``, else $HV_TUNE_CACHE, else
        ~/.cache/hv_tiles.json) keyed by the padded grid, shot count and k, and
        reused when present (the key includes the menu size, so a library with a
        different menu tunes again)."""
        import json
        import os
        path = cache or os.environ.get("HV_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                                       "hv_tiles.json")
        key = f"{self.NZ}x{self.NX}/ns{self.ns}/k{int(k)}/menu{menu_size()}"
        try:
            table = json.load(open(path))
        except Exception:
            table = {}
        if key in table:
            self.set_tiles(table[key])
            return tuple(table[key])
        ws, nb = self._workspace(HV_OP_HV, k, 1)
        chosen = (ctypes.c_int * 3)()
        check(self.lib.hv_autotune(self._h, int(k), ws, nb, self._stream(), chosen, None))
        table[key] = list(chosen)
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = f"{path}.{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass
        return tuple(chosen)

    # ---------------------------------------------------------------- workspace
    def workspace_size(self, op: int, k: int = 1, ckpt: int = HV_CKPT_ALL) -> int:
        n = ctypes.c_size_t()
        check(self.lib.hv_workspace_size(self._h, op, int(k), int(ckpt), ctypes.byref(n)))
        return n.value

    def _workspace(self, op, k, ckpt):
        need = self.workspace_size(op, k, ckpt)
        buf = self._ws.get("ws")
        if buf is None or buf.numel() < need:
            self._ws.pop("ws", None)
            buf = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            self._ws["ws"] = buf
        return buf.data_ptr(), buf.numel()

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _m(self, m):
        return _dev(m, torch.float32, (self.nz, self.nx), "m", self.device)

    # ---------------------------------------------------------------- operations
    def fwd_model(self, m: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """d[ns, nt, nr] = f(m) (paper eq. (data) without noise)."""
        d = out if out is not None else torch.empty((self.ns, self.nt, self.nr), dtype=torch.float32, device=self.device)
        pm, pd = self._m(m), _dev(d, torch.float32, (self.ns, self.nt, self.nr), "d", self.device)
        ws, nb = self._workspace(HV_OP_FWD, 1, HV_CKPT_ALL)
        check(self.lib.hv_fwd_model(self._h, pm, pd, ws, nb, self._stream()))
        return d

    def wavefield(self, m: torch.Tensor, steps) -> torch.Tensor:
        """u^{n+1} of every shot on the padded grid at the given steps n: [len(steps), ns, NZ, NX]."""
        steps = _i32(steps)
        out = torch.empty((steps.size, self.ns, self.NZ, self.NX), dtype=torch.float32, device=self.device)
        ws, nb = self._workspace(HV_OP_WAVEFIELD, 1, HV_CKPT_ALL)
        check(self.lib.hv_wavefield(self._h, self._m(m), int(steps.size), steps.ctypes.data_as(_lib.ip),
                                    out.data_ptr(), ws, nb, self._stream()))
        return out

    def born(self, m: torch.Tensor, dm: torch.Tensor) -> torch.Tensor:
        """F dm for dm[k, nz, nx] -> [k, ns, nt, nr]."""
        k = dm.shape[0]
        pdm = _dev(dm, torch.float32, (k, self.nz, self.nx), "dm", self.device)
        dd = torch.empty((k, self.ns, self.nt, self.nr), dtype=torch.float32, device=self.device)
        ws, nb = self._workspace(HV_OP_BORN, k, HV_CKPT_ALL)
        check(self.lib.hv_born(self._h, self._m(m), pdm, k, dd.data_ptr(), ws, nb, self._stream()))
        return dd

    def migrate(self, m: torch.Tensor, r: torch.Tensor, ckpt: int = HV_CKPT_ALL) -> torch.Tensor:
        """F^T r for data r[ns, nt, nr] -> [nz, nx]."""
        pr = _dev(r, torch.float32, (self.ns, self.nt, self.nr), "r", self.device)
        g = torch.empty((self.nz, self.nx), dtype=torch.float32, device=self.device)
        ws, nb = self._workspace(HV_OP_MIGRATE, 1, ckpt)
        check(self.lib.hv_migrate(self._h, self._m(m), pr, g.data_ptr(), int(ckpt), ws, nb, self._stream()))
        return g

    def misfit_grad(self, m: torch.Tensor, d_obs: torch.Tensor, ckpt: int = HV_CKPT_ALL):
        """(phi, grad): phi a 0-d float64 CUDA tensor, grad [nz, nx]."""
        pd = _dev(d_obs, torch.float32, (self.ns, self.nt, self.nr), "d_obs", self.device)
        phi = torch.empty((), dtype=torch.float64, device=self.device)
        g = torch.empty((self.nz, self.nx), dtype=torch.float32, device=self.device)
        ws, nb = self._workspace(HV_OP_GRAD, 1, ckpt)
        check(self.lib.hv_misfit_grad(self._h, self._m(m), pd, phi.data_ptr(), g.data_ptr(), int(ckpt), ws, nb,
                                      self._stream()))
        return phi, g

    def misfit(self, m: torch.Tensor, d_obs: torch.Tensor) -> torch.Tensor:
        """phi = 1/(2 sigma^2) sum (f(m) - d_obs)^2 as a 0-d float64 CUDA tensor (hv_misfit)."""
        pd = _dev(d_obs, torch.float32, (self.ns, self.nt, self.nr), "d_obs", self.device)
        phi = torch.empty((), dtype=torch.float64, device=self.device)
        ws, nb = self._workspace(_lib.HV_OP_MISFIT, 1, HV_CKPT_ALL)
        check(self.lib.hv_misfit(self._h, self._m(m), pd, phi.data_ptr(), ws, nb, self._stream()))
        return phi

    def misfit_models(self, ms: torch.Tensor, d_obs: torch.Tensor) -> torch.Tensor:
        """phi[i] = 1/(2 sigma^2) sum (f(ms[i]) - d_obs)^2 for the k models ms [k, nz, nx] in one forward sweep
        (hv_misfit_models); d_obs is [ns, nt, nr] for every model or [k, ns, nt, nr].  Returns a float64 CUDA
        tensor [k], each entry bitwise misfit(ms[i], d_obs[i])."""
        if not isinstance(ms, torch.Tensor) or ms.dim() != 3:
            raise ValueError("ms: expected a [k, nz, nx] tensor")
        k = ms.shape[0]
        pm = _dev(ms, torch.float32, (k, self.nz, self.nx), "ms", self.device)
        shared = isinstance(d_obs, torch.Tensor) and d_obs.dim() == 3
        pd = _dev(d_obs, torch.float32, (self.ns, self.nt, self.nr) if shared else (k, self.ns, self.nt, self.nr),
                  "d_obs", self.device)
        phi = torch.empty(k, dtype=torch.float64, device=self.device)
        nd, npt = self.ns * self.nt * self.nr * 4, self.nz * self.nx * 4
        arr = ctypes.c_void_p * max(k, 1)
        m_p = arr(*[pm + i * npt for i in range(k)])
        d_p = arr(*[pd + (0 if shared else i * nd) for i in range(k)])
        f_p = arr(*[phi.data_ptr() + 8 * i for i in range(k)])
        ws, nb = self._workspace(_lib.HV_OP_MISFITS, k, HV_CKPT_ALL)
        check(self.lib.hv_misfit_models(self._h, int(k), m_p, d_p, f_p, ws, nb, self._stream()))
        return phi

    def set_highpass(self, rho_c: float) -> None:
        """PSF and PDO builds on this problem approximate F_hp H_d F_hp (rho_c > 0 [rad/m]) or H_d (0)
        (hv_set_highpass)."""
        check(self.lib.hv_set_highpass(self._h, float(rho_c)))

    def set_image_precision(self, mode: int) -> None:
        """Imaging sum: HV_IMAGE_PAIRS (default) or the FP64 check HV_IMAGE_FP64 (hv_set_image_precision)."""
        check(self.lib.hv_set_image_precision(self._h, int(mode)))

    def set_wait_limit(self, seconds: float) -> None:
        """Limit of every bounded device wait of this problem's kernels (hv_set_wait_limit)."""
        check(self.lib.hv_set_wait_limit(self._h, float(seconds)))

    def inject_wait_timeout(self) -> None:
        """Make the next dataflow-ordered stencil step's waits run out (hv_inject_wait_timeout; testing)."""
        check(self.lib.hv_inject_wait_timeout(self._h))

    def hessian_apply(self, m: torch.Tensor, v: torch.Tensor, ckpt: int = HV_CKPT_ALL,
                      out_dtype=torch.float32) -> torch.Tensor:
        """H_d v for v[k, nz, nx] -> [k, nz, nx] (float32 or float64 output)."""
        k = v.shape[0]
        pv = _dev(v, torch.float32, (k, self.nz, self.nx), "v", self.device)
        out = torch.empty((k, self.nz, self.nx), dtype=out_dtype, device=self.device)
        ws, nb = self._workspace(HV_OP_HV, k, ckpt)
        fn = self.lib.hv_hessian_apply if out_dtype == torch.float32 else self.lib.hv_hessian_apply_f64out
        if out_dtype not in (torch.float32, torch.float64):
            raise ValueError("out_dtype must be float32 or float64")
        check(fn(self._h, self._m(m), pv, k, out.data_ptr(), int(ckpt), ws, nb, self._stream()))
        return out


    def apply_batch(self, m: torch.Tensor, hv=(), grads=(), misfits=(), ckpt: int = HV_CKPT_ALL):
        """One merged call at model m (hv_apply_batch): H v for each v[k, nz, nx] in ``hv``, (phi, gradient)
        for each observed data set in ``grads``, phi for each in ``misfits``; every result bitwise that of
        the separate call.  Returns (list of H v, list of (phi, grad), list of phi)."""
        hv, grads, misfits = list(hv), list(grads), list(misfits)
        dshape = (self.ns, self.nt, self.nr)
        pv = [_dev(v, torch.float32, (v.shape[0], self.nz, self.nx), "v", self.device) for v in hv]
        outs = [torch.empty(v.shape, dtype=torch.float32, device=self.device) for v in hv]
        pg = [_dev(d, torch.float32, dshape, "d_obs", self.device) for d in grads]
        gphi = [torch.empty((), dtype=torch.float64, device=self.device) for _ in grads]
        gout = [torch.empty((self.nz, self.nx), dtype=torch.float32, device=self.device) for _ in grads]
        pm = [_dev(d, torch.float32, dshape, "d_obs", self.device) for d in misfits]
        mphi = [torch.empty((), dtype=torch.float64, device=self.device) for _ in misfits]

        def arr(ptrs, t=ctypes.c_void_p):
            return (t * max(len(ptrs), 1))(*ptrs)

        keep = [arr(pv), arr([v.shape[0] for v in hv], ctypes.c_int), arr([o.data_ptr() for o in outs]),
                arr(pg), arr([x.data_ptr() for x in gphi]), arr([x.data_ptr() for x in gout]),
                arr(pm), arr([x.data_ptr() for x in mphi])]
        b = _lib.HvBatch(len(hv), keep[0], keep[1], keep[2], len(grads), keep[3], keep[4], keep[5],
                         len(misfits), keep[6], keep[7])
        n = ctypes.c_size_t()
        check(self.lib.hv_batch_workspace_size(self._h, ctypes.byref(b), int(ckpt), ctypes.byref(n)))
        buf = self._ws.get("ws")
        if buf is None or buf.numel() < n.value:
            self._ws.pop("ws", None)
            buf = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._ws["ws"] = buf
        check(self.lib.hv_apply_batch(self._h, self._m(m), ctypes.byref(b), int(ckpt), buf.data_ptr(), buf.numel(),
                                      self._stream()))
        return outs, list(zip(gphi, gout)), mphi

    def hessian_apply_partial(self, m: torch.Tensor, v: torch.Tensor, ckpt: int = HV_CKPT_ALL) -> torch.Tensor:
        """The extended image of this problem's shots before the fold, [k, NZ, NX] float64
        (hv_hessian_apply_partial); sum it over shot blocks, then fold."""
        k = v.shape[0]
        pv = _dev(v, torch.float32, (k, self.nz, self.nx), "v", self.device)
        ext = torch.empty((k, self.NZ, self.NX), dtype=torch.float64, device=self.device)
        ws, nb = self._workspace(HV_OP_HV, k, ckpt)
        check(self.lib.hv_hessian_apply_partial(self._h, self._m(m), pv, k, ext.data_ptr(), int(ckpt), ws, nb,
                                                self._stream()))
        return ext

    def fold(self, ext: torch.Tensor, out_dtype=torch.float32) -> torch.Tensor:
        """E^T of extended images [k, NZ, NX] float64 -> [k, nz, nx] (hv_image_fold)."""
        k = ext.shape[0]
        pe = _dev(ext, torch.float64, (k, self.NZ, self.NX), "ext", self.device)
        out = torch.empty((k, self.nz, self.nx), dtype=out_dtype, device=self.device)
        if out_dtype == torch.float32:
            check(self.lib.hv_image_fold(self._h, pe, k, out.data_ptr(), None, self._stream()))
        elif out_dtype == torch.float64:
            check(self.lib.hv_image_fold(self._h, pe, k, None, out.data_ptr(), self._stream()))
        else:
            raise ValueError("out_dtype must be float32 or float64")
        return out

    # ---------------------------------------------------------------- approximations
    def approx_build_psf(self, m: torch.Tensor, spacing: int, n_batches: int = 4,
                         ckpt: int = HV_CKPT_ALL) -> "PsfApprox":
        """Point-spread-function approximation of H_d at m (hv_approx_build_psf): n_batches = B*B
        Hessian applications to impulse lattices of spacing `spacing` cells."""
        n = ctypes.c_size_t()
        check(self.lib.hv_approx_psf_workspace_size(self._h, int(n_batches), int(ckpt), ctypes.byref(n)))
        buf = self._ws.get("ws")
        if buf is None or buf.numel() < n.value:
            self._ws.pop("ws", None)
            buf = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._ws["ws"] = buf
        out = ctypes.c_void_p()
        check(self.lib.hv_approx_build_psf(self._h, self._m(m), int(spacing), int(n_batches), int(ckpt),
                                           ctypes.byref(out), buf.data_ptr(), buf.numel(), self._stream()))
        return PsfApprox(self.lib, out, self.device)

    def approx_build_lr(self, m: torch.Tensor, delta: float, gamma: float, rank: int, omega: torch.Tensor,
                        ckpt: int = HV_CKPT_ALL) -> "LrApprox":
        """Low-rank approximation (hv_approx_build_lr): the `rank` leading eigenpairs of H_d v = lambda R v
        with the Matern prior R = (delta I - gamma Lap)^2, from the test matrix omega [k, nz, nx]."""
        k = omega.shape[0]
        po = _dev(omega, torch.float32, (k, self.nz, self.nx), "omega", self.device)
        n = ctypes.c_size_t()
        check(self.lib.hv_approx_lr_workspace_size(self._h, int(k), int(ckpt), ctypes.byref(n)))
        buf = self._ws.get("ws")
        if buf is None or buf.numel() < n.value:
            self._ws.pop("ws", None)
            buf = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._ws["ws"] = buf
        out = ctypes.c_void_p()
        check(self.lib.hv_approx_build_lr(self._h, self._m(m), float(delta), float(gamma), int(rank), po, int(k),
                                          int(ckpt), ctypes.byref(out), buf.data_ptr(), buf.numel(), self._stream()))
        return LrApprox(self.lib, out, self.device)

    def approx_build_pdo(self, m: torch.Tensor, rho0: float, r: int = 8, ckpt: int = HV_CKPT_ALL) -> "PdoApprox":
        """Pseudo-differential-operator probing approximation of H_d at m (hv_approx_build_pdo): one
        Hessian application to r sinusoids on the circle of radius rho0 [rad/m]."""
        n = ctypes.c_size_t()
        check(self.lib.hv_approx_pdo_workspace_size(self._h, int(ckpt), ctypes.byref(n)))
        buf = self._ws.get("ws")
        if buf is None or buf.numel() < n.value:
            self._ws.pop("ws", None)
            buf = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            self._ws["ws"] = buf
        out = ctypes.c_void_p()
        check(self.lib.hv_approx_build_pdo(self._h, self._m(m), float(rho0), int(r), int(ckpt), ctypes.byref(out),
                                           buf.data_ptr(), buf.numel(), self._stream()))
        return PdoApprox(self.lib, out, self.device)


class MisfitEngine:
    """Misfits that join a running forward sweep at its next time step (hv_engine_*): `slots` models, each with
    its own step counter, advanced together one time step per tick.  All work runs on the problem's stream (the
    current torch stream)."""

    def __init__(self, problem: Problem, slots: int):
        self.P, self.lib, self.slots = problem, problem.lib, int(slots)
        n = ctypes.c_size_t()
        check(self.lib.hv_engine_workspace_size(problem._h, self.slots, ctypes.byref(n)))
        self._ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=problem.device)
        e = ctypes.c_void_p()
        check(self.lib.hv_engine_create(problem._h, self.slots, self._ws.data_ptr(), self._ws.numel(), ctypes.byref(e)))
        self._e = e
        self._done = (ctypes.c_int * self.slots)()
        self._held = {}                 # slot -> the tensors its work reads and writes

    def join(self, m: torch.Tensor, d_obs: torch.Tensor):
        """(slot, phi): phi (0-d float64) receives the misfit once the slot is reported done by tick()."""
        P = self.P
        pm = P._m(m)
        pd = _dev(d_obs, torch.float32, (P.ns, P.nt, P.nr), "d_obs", P.device)
        phi = torch.empty((), dtype=torch.float64, device=P.device)
        slot = ctypes.c_int()
        check(self.lib.hv_engine_join(self._e, pm, pd, phi.data_ptr(), P._stream(), ctypes.byref(slot)))
        self._held[slot.value] = (m, d_obs, phi)
        return slot.value, phi

    def tick(self) -> list:
        """One time step of every occupied slot; returns the slots whose misfit this tick completed."""
        n = ctypes.c_int()
        check(self.lib.hv_engine_tick(self._e, self.P._stream(), self._done, ctypes.byref(n)))
        done = [self._done[i] for i in range(n.value)]
        for j in done:
            self._held.pop(j, None)
        return done

    @property
    def active(self) -> int:
        n = ctypes.c_int()
        check(self.lib.hv_engine_active(self._e, ctypes.byref(n)))
        return n.value

    # ---- the device-resident loop (hv_engine_post / serve / poll / stop)
    def post(self, m: torch.Tensor, d_obs: torch.Tensor, stream=None):
        """(slot, phi): the request is prepared and posted on `stream` (default: the current stream); the
        running loop admits it at its next time step.  phi is written once poll() reports the slot."""
        P = self.P
        pm = P._m(m)
        pd = _dev(d_obs, torch.float32, (P.ns, P.nt, P.nr), "d_obs", P.device)
        phi = torch.empty((), dtype=torch.float64, device=P.device)
        s = stream if stream is not None else torch.cuda.current_stream(P.device)
        slot = ctypes.c_int()
        check(self.lib.hv_engine_post(self._e, pm, pd, phi.data_ptr(), ctypes.c_void_p(s.cuda_stream),
                                      ctypes.byref(slot)))
        self._held[slot.value] = (m, d_obs, phi)
        return slot.value, phi

    def serve(self, stream) -> None:
        """Launch the loop on `stream` (a torch.cuda.Stream) unless it is running."""
        check(self.lib.hv_engine_serve(self._e, ctypes.c_void_p(stream.cuda_stream)))

    def poll(self):
        """(done slots, running): the slots whose misfit is written since the last poll, and whether the loop
        is running."""
        n, run = ctypes.c_int(), ctypes.c_int()
        check(self.lib.hv_engine_poll(self._e, self._done, ctypes.byref(n), ctypes.byref(run)))
        done = [self._done[i] for i in range(n.value)]
        for j in done:
            self._held.pop(j, None)
        return done, bool(run.value)

    def stop(self) -> None:
        """Ask the running loop to end after its current iteration."""
        check(self.lib.hv_engine_stop(self._e))

    def close(self) -> None:
        if getattr(self, "_e", None):
            self.lib.hv_engine_destroy(self._e)          # ends a running loop
            torch.cuda.synchronize(self.P.device)        # posts and ticks on any stream, before the workspace goes
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Approx:
    """A built Hessian approximation (owns its device memory; see hv_approx_*)."""

    def __init__(self, lib, handle, device):
        self.lib, self._a, self.device = lib, handle, device
        info = (ctypes.c_int * 11)()
        check(self.lib.hv_approx_info(self._a, info))
        keys = ("kind", "r", "R", "na", "nb", "S", "B", "cz0", "cx0", "nz", "nx")
        self.info = dict(zip(keys, list(info)))
        if self.info["kind"] in (1, 2):
            self.info["spd"] = self.info.pop("R")

    def apply(self, v: torch.Tensor, mode: int = 0) -> torch.Tensor:
        """H~ v (mode 0 = HV_APPROX_H) or the mode's operator for v[k, nz, nx] -> [k, nz, nx] (hv_approx_apply)."""
        nz, nx = self.info["nz"], self.info["nx"]
        k = v.shape[0]
        pv = _dev(v, torch.float32, (k, nz, nx), "v", self.device)
        out = torch.empty((k, nz, nx), dtype=torch.float32, device=self.device)
        check(self.lib.hv_approx_apply(self._a, pv, k, out.data_ptr(), int(mode),
                                       ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))
        return out

    def close(self):
        if getattr(self, "_a", None):
            self.lib.hv_approx_destroy(self._a)
            self._a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PsfApprox(Approx):
    """Point-spread-function approximation (hv_approx_build_psf)."""

    def psfs(self) -> torch.Tensor:
        """The PSFs [r, 2R+1, 2R+1] (a device copy)."""
        W = 2 * self.info["R"] + 1
        out = torch.empty((self.info["r"], W, W), dtype=torch.float32, device=self.device)
        check(self.lib.hv_approx_psfs(self._a, out.data_ptr(),
                                      ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))
        return out


class PdoApprox(Approx):
    """A low-rank-symbol approximation: PDO probing (hv_approx_build_pdo) or PSF+ (psf_plus)."""

    def symbol(self):
        """(a, b): the symbol factors [r, nz, nx] complex64 each (b in DFT order), device copies."""
        r, nz, nx = self.info["r"], self.info["nz"], self.info["nx"]
        a = torch.empty((r, nz, nx, 2), dtype=torch.float32, device=self.device)
        b = torch.empty((r, nz, nx, 2), dtype=torch.float32, device=self.device)
        check(self.lib.hv_approx_pdo_symbol(self._a, a.data_ptr(), b.data_ptr(),
                                            ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))
        return torch.view_as_complex(a), torch.view_as_complex(b)

    def sqrt(self) -> "PdoApprox":
        """The square-root form (section 3.7) of a PDO approximation (hv_approx_sqrt_pdo): apply gives
        B B^T v, apply(v, HV_APPROX_SQRT) B v and apply(v, HV_APPROX_SQRT_T) B^T v."""
        out = ctypes.c_void_p()
        check(self.lib.hv_approx_sqrt_pdo(self._a, ctypes.byref(out),
                                          ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))
        return PdoApprox(self.lib, out, self.device)


class LrApprox(Approx):
    """Low-rank approximation with the Matern prior (hv_approx_build_lr)."""

    def eigs(self):
        """(lambda [rank] float64 numpy, V [rank, nz, nx] device tensor) of H_d v = lambda R v."""
        r, nz, nx = self.info["r"], self.info["nz"], self.info["nx"]
        lam = np.empty(r)
        V = torch.empty((r, nz, nx), dtype=torch.float32, device=self.device)
        check(self.lib.hv_approx_lr_eigs(self._a, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), V.data_ptr(),
                                         ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))
        return lam, V

    def sample_factor(self, n: torch.Tensor) -> torch.Tensor:
        """(I - V S V^T R) A^-1 n: maps N(0, I) draws to the Laplace approximation N(0, (H~_d + R)^-1)."""
        return self.apply(n, mode=2)


def prior_apply(v: torch.Tensor, h: float, delta: float, gamma: float, op: int) -> torch.Tensor:
    """A v (op 0), A^-1 v (1), R v (2) or R^-1 v (3) for the Matern prior, v [k, nz, nx] (hv_prior_apply)."""
    k, nz, nx = v.shape
    pv = _dev(v, torch.float32, (k, nz, nx), "v", v.device)
    out = torch.empty_like(v, dtype=torch.float32)
    check(_lib.load().hv_prior_apply(nz, nx, float(h), float(delta), float(gamma), pv, k, out.data_ptr(), int(op),
                                     ctypes.c_void_p(torch.cuda.current_stream(v.device).cuda_stream)))
    return out


def count_nonfinite(x: torch.Tensor) -> int:
    """Number of NaN and +-Inf entries of a float32 CUDA tensor (hv_count_nonfinite)."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("x: expected a contiguous float32 CUDA tensor")
    lib = _lib.load()
    cnt = torch.empty((), dtype=torch.int64, device=x.device)
    check(lib.hv_count_nonfinite(x.data_ptr(), x.numel(), cnt.data_ptr(),
                                 ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)))
    return int(cnt)


def highpass_apply(v: torch.Tensor, h: float, rho_c: float) -> torch.Tensor:
    """F_hp v = Re F^-1 (phi(|xi|) F v), phi(rho) = 1 - exp(-rho^2 / (2 rho_c^2)), for v [k, nz, nx]
    (hv_highpass_apply): the high-pass filter applied before the PSF and PDO approximations."""
    k, nz, nx = v.shape
    pv = _dev(v, torch.float32, (k, nz, nx), "v", v.device)
    out = torch.empty_like(v, dtype=torch.float32)
    check(_lib.load().hv_highpass_apply(nz, nx, float(h), float(rho_c), pv, k, out.data_ptr(),
                                        ctypes.c_void_p(torch.cuda.current_stream(v.device).cuda_stream)))
    return out


class Filtered:
    """F_hp Op F_hp for the operator of `src` (an object with .operator(), .device, .lib, e.g. Quad): the
    filtered operator the PSF and PDO approximations are built from (hv_filtered_*).  Keeps `src` alive."""

    def __init__(self, src, rho_c: float, max_k: int = 64):
        self.lib, self.device, self.src = src.lib, src.device, src
        f = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hv_filtered_create(ctypes.byref(src.operator()), float(rho_c), int(max_k), ctypes.byref(f)))
        self._f = f
        self._op = _lib.HvOperator()
        check(self.lib.hv_filtered_operator(self._f, ctypes.byref(self._op)))

    def operator(self):
        return self._op

    def close(self):
        if getattr(self, "_f", None):
            self.lib.hv_filtered_destroy(self._f)
            self._f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def psf_plus(psf: PsfApprox, pdo: PdoApprox, tol: float = 1e-3, spd: bool = False) -> PdoApprox:
    """PSF+ (hv_approx_build_psfplus): the PSF symbol rows' dominant directions refined
    against the PDO symbol columns; the result is a low-rank-symbol approximation.  spd: the
    square-root form of section 3.7 (hv_approx_build_psfplus_sqrt), applied as B B^T."""
    out = ctypes.c_void_p()
    fn = psf.lib.hv_approx_build_psfplus_sqrt if spd else psf.lib.hv_approx_build_psfplus
    check(fn(psf._a, pdo._a, float(tol), ctypes.byref(out),
             ctypes.c_void_p(torch.cuda.current_stream(psf.device).cuda_stream)))
    return PdoApprox(psf.lib, out, psf.device)


class Quad:
    """The ideal quadratic test model of section 4.1 on one GPU (hv_quad_*): misfit Hessian
    W (A A^T + V Lambda V^T) W, A the order-1/2 PsiDO of the rank-3 symbol, and the objective
    Phi(m) = 1/2 (W m - m*)^T H_d (W m - m*) + 1/2 m^T R m with the Matern prior (delta, gamma)."""

    def __init__(self, nz: int, nx: int, h: float, lam, delta: float, gamma: float, rho_c: float | None = None,
                 taper: int | None = None, device=None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.nz, self.nx, self.h = int(nz), int(nx), float(h)
        self.rho_c = np.pi / (2 * h) if rho_c is None else float(rho_c)
        self.taper = max(1, min(nz, nx) // 8) if taper is None else int(taper)
        self.lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
        self.delta, self.gamma = float(delta), float(gamma)
        q = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hv_quad_create(self.nz, self.nx, self.h, self.rho_c, self.taper, len(self.lam),
                                          self.lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.delta,
                                          self.gamma, ctypes.byref(q)))
        self._q = q
        self._op = _lib.HvOperator()
        check(self.lib.hv_quad_operator(self._q, ctypes.byref(self._op)))

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def apply(self, v: torch.Tensor, op: int = _lib.HV_QUAD_HD) -> torch.Tensor:
        k = v.shape[0]
        pv = _dev(v, torch.float32, (k, self.nz, self.nx), "v", self.device)
        out = torch.empty((k, self.nz, self.nx), dtype=torch.float32, device=self.device)
        check(self.lib.hv_quad_apply(self._q, int(op), pv, k, out.data_ptr(), self._stream()))
        return out

    def objective(self, m: torch.Tensor, mstar: torch.Tensor, grad: bool = True):
        """(phi [k] float64 device, grad [k, nz, nx] or None) for states m [k, nz, nx]; mstar [nz, nx] or [k, nz, nx]."""
        k = m.shape[0]
        pm = _dev(m, torch.float32, (k, self.nz, self.nx), "m", self.device)
        one = mstar.dim() == 2
        ps = _dev(mstar, torch.float32, (self.nz, self.nx) if one else (k, self.nz, self.nx), "mstar", self.device)
        phi = torch.empty(k, dtype=torch.float64, device=self.device)
        g = torch.empty((k, self.nz, self.nx), dtype=torch.float32, device=self.device) if grad else None
        check(self.lib.hv_quad_objective(self._q, pm, ps, k, int(one), phi.data_ptr(),
                                         g.data_ptr() if grad else None, self._stream()))
        return phi, g

    def tables(self):
        """(a [3, nz, nx] complex, b [3, nz, nx] complex (DFT order), V [nlr, nz, nx], W [nz, nx]) device copies."""
        N = (self.nz, self.nx)
        a = torch.empty((3, *N, 2), dtype=torch.float32, device=self.device)
        b = torch.empty((3, *N, 2), dtype=torch.float32, device=self.device)
        V = torch.empty((len(self.lam), *N), dtype=torch.float32, device=self.device)
        W = torch.empty(N, dtype=torch.float32, device=self.device)
        check(self.lib.hv_quad_tables(self._q, a.data_ptr(), b.data_ptr(), V.data_ptr() if len(self.lam) else None,
                                      W.data_ptr(), self._stream()))
        return torch.view_as_complex(a), torch.view_as_complex(b), V, W

    def operator(self):
        """The misfit Hessian as an hv_operator (for the *_op approximation builds)."""
        return self._op

    def close(self):
        if getattr(self, "_q", None):
            self.lib.hv_quad_destroy(self._q)
            self._q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _op_stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def approx_build_psf_op(src, spacing: int, n_batches: int = 4) -> PsfApprox:
    """PSF approximation of the operator of `src` (an object with .operator(), .device, e.g. Quad)."""
    out = ctypes.c_void_p()
    check(src.lib.hv_approx_build_psf_op(ctypes.byref(src.operator()), int(spacing), int(n_batches), ctypes.byref(out),
                                         _op_stream(src.device)))
    return PsfApprox(src.lib, out, src.device)


def approx_build_pdo_op(src, rho0: float, r: int = 8) -> PdoApprox:
    """PDO approximation of the operator of `src`."""
    out = ctypes.c_void_p()
    check(src.lib.hv_approx_build_pdo_op(ctypes.byref(src.operator()), float(rho0), int(r), ctypes.byref(out),
                                         _op_stream(src.device)))
    return PdoApprox(src.lib, out, src.device)


def approx_build_lr_op(src, delta: float, gamma: float, rank: int, omega: torch.Tensor) -> LrApprox:
    """Low-rank approximation of the operator of `src` with the Matern prior (delta, gamma)."""
    op = src.operator()
    k = omega.shape[0]
    po = _dev(omega, torch.float32, (k, op.nz, op.nx), "omega", src.device)
    out = ctypes.c_void_p()
    check(src.lib.hv_approx_build_lr_op(ctypes.byref(op), float(delta), float(gamma), int(rank), po, int(k),
                                        ctypes.byref(out), _op_stream(src.device)))
    return LrApprox(src.lib, out, src.device)


class Posterior:
    """Laplace approximation H~ = H~_d + R (+ a low-rank correction) of the posterior (hv_posterior_*):
    H~_d = B B^T from a square-root approximation `approx` (or 0), R the Matern prior (delta, gamma)."""

    def __init__(self, nz: int, nx: int, h: float, delta: float, gamma: float, approx: "Approx | None" = None,
                 device=None, max_k: int = 64):
        self.lib = _lib.load()
        self.device = (approx.device if approx is not None else
                       torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device))
        self.nz, self.nx = int(nz), int(nx)
        self.approx = approx                      # kept alive: the posterior borrows it
        p = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hv_posterior_create(self.nz, self.nx, float(h), float(delta), float(gamma),
                                               approx._a if approx is not None else None, int(max_k),
                                               ctypes.byref(p)))
        self._p = p

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _f(self, t, name, k=None):
        k = t.shape[0] if k is None else k
        return _dev(t, torch.float32, (k, self.nz, self.nx), name, self.device)

    def solve(self, b: torch.Tensor, op=None, rtol: float = 1e-6, max_iter: int = 1000):
        """(x, iterations): x = (Op + R)^-1 b, Op = op.operator() of an operator source or H~_d."""
        k = b.shape[0]
        x = torch.empty_like(b)
        it = ctypes.c_int()
        opp = ctypes.byref(op.operator()) if op is not None else None
        check(self.lib.hv_posterior_solve(self._p, opp, self._f(b, "b"), k, x.data_ptr(), float(rtol), int(max_iter),
                                          ctypes.byref(it), self._stream()))
        return x, it.value

    def apply(self, v: torch.Tensor) -> torch.Tensor:
        out = torch.empty_like(v)
        check(self.lib.hv_posterior_apply(self._p, self._f(v, "v"), v.shape[0], out.data_ptr(), self._stream()))
        return out

    def sample(self, n1: torch.Tensor, n2: torch.Tensor | None = None, rtol: float = 1e-6, max_iter: int = 1000):
        """(zeta, iterations): zeta ~ N(0, H~^-1) from standard normals n1, n2 [k, nz, nx]."""
        k = n1.shape[0]
        zeta = torch.empty_like(n1)
        it = ctypes.c_int()
        p2 = self._f(n2, "n2", k) if n2 is not None else None
        check(self.lib.hv_posterior_sample(self._p, self._f(n1, "n1"), p2, k, zeta.data_ptr(), float(rtol),
                                           int(max_iter), ctypes.byref(it), self._stream()))
        return zeta, it.value

    def correct(self, src, omega: torch.Tensor, rank: int, rtol: float = 1e-6, max_iter: int = 1000):
        """Low-rank correction against the operator of `src` (e.g. Quad) with test matrix omega [k, nz, nx]."""
        k = omega.shape[0]
        check(self.lib.hv_posterior_correct(self._p, ctypes.byref(src.operator()), self._f(omega, "omega"), k,
                                            int(rank), float(rtol), int(max_iter), self._stream()))

    def eigs(self):
        r = self.lib.hv_posterior_rank(self._p)
        lam = np.empty(r)
        V = torch.empty((r, self.nz, self.nx), dtype=torch.float32, device=self.device)
        check(self.lib.hv_posterior_eigs(self._p, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         V.data_ptr() if r else None, self._stream()))
        return lam, V

    def close(self):
        if getattr(self, "_p", None):
            self.lib.hv_posterior_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gpcn_propose(m: torch.Tensor, m_map: torch.Tensor, zeta: torch.Tensor, beta: float):
    """(m_new, d_new = m_new - m_map) for chains m [c, nz, nx] (hv_gpcn_propose)."""
    c = m.shape[0]
    n = m[0].numel()
    m_new, d_new = torch.empty_like(m), torch.empty_like(m)
    check(_lib.load().hv_gpcn_propose(n, c, m.data_ptr(), m_map.data_ptr(), zeta.data_ptr(), float(beta),
                                      m_new.data_ptr(), d_new.data_ptr(),
                                      ctypes.c_void_p(torch.cuda.current_stream(m.device).cuda_stream)))
    return m_new, d_new


def gpcn_accept(phi_new: torch.Tensor, m_new: torch.Tensor, d_new: torch.Tensor, Hd_new: torch.Tensor,
                log_u: torch.Tensor, m: torch.Tensor, delta_cur: torch.Tensor) -> torch.Tensor:
    """Accept/reject every chain (hv_gpcn_accept); updates m and delta_cur in place, returns accepted [c] int32."""
    c = m.shape[0]
    for t, dt in ((phi_new, torch.float64), (log_u, torch.float64), (delta_cur, torch.float64)):
        if t.dtype != dt or t.shape != (c,) or not t.is_cuda:
            raise ValueError("phi_new, log_u, delta_cur: float64 [c] CUDA tensors")
    acc = torch.empty(c, dtype=torch.int32, device=m.device)
    check(_lib.load().hv_gpcn_accept(m[0].numel(), c, phi_new.data_ptr(), m_new.data_ptr(), d_new.data_ptr(),
                                     Hd_new.data_ptr(), log_u.data_ptr(), m.data_ptr(), delta_cur.data_ptr(),
                                     acc.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream(m.device).cuda_stream)))
    return acc


def hermitian_eig(A: np.ndarray):
    """(w descending, V) of a Hermitian matrix by the library's host Jacobi routine (hv_util_hermitian_eig)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n), dtype=np.complex128)
    dp = ctypes.POINTER(ctypes.c_double)
    check(_lib.load().hv_util_hermitian_eig(n, A.view(np.float64).ctypes.data_as(dp), w.ctypes.data_as(dp),
                                            V.view(np.float64).ctypes.data_as(dp)))
    return w, V


def set_fused_transforms(enable: bool = True) -> None:
    """Fused low-rank-symbol transforms for approximations created afterwards (hv_set_fused_transforms)."""
    check(_lib.load().hv_set_fused_transforms(int(bool(enable))))


def checkpoint_schedule(nt: int, slots: int):
    """The library's checkpoint schedule: (actions[n, 3] int32, recomputed forward steps)."""
    lib = _lib.load()
    n = ctypes.c_int()
    adv = ctypes.c_longlong()
    check(lib.hv_checkpoint_schedule(int(nt), int(slots), None, 0, ctypes.byref(n), ctypes.byref(adv)))
    acts = np.zeros((n.value, 3), dtype=np.int32)
    check(lib.hv_checkpoint_schedule(int(nt), int(slots), acts.ctypes.data_as(_lib.ip), n.value, ctypes.byref(n),
                                     ctypes.byref(adv)))
    return acts, adv.value


def kernel_launches() -> int:
    """Kernels launched by libhv in this process so far."""
    return int(_lib.load().hv_kernel_launches())


def menu_size() -> int:
    """Number of tile configurations the stencil kernels come in."""
    return int(_lib.load().hv_tile_menu_size())


def menu_info(index: int) -> dict:
    """Tile shape, threads, copy stages and 8-shot groups per CTA of a menu entry."""
    info = (ctypes.c_int * 5)()
    check(_lib.load().hv_tile_menu_info(int(index), info))
    return {"TX": info[0], "TZ": info[1], "threads": info[2], "stages": info[3], "groups_per_cta": info[4]}
