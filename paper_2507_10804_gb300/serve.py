"""Python face of the request server (hv_server_*): submit H v, gradient and
misfit requests from many clients; the library's scheduler admits them by
device-memory budget, merges queued requests on one problem and model into
one call, and runs them concurrently on its streams.

Tensors passed to ``submit`` are kept alive by the server object until the
request is done.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import HV_REQ_APPROX, HV_REQ_GRAD, HV_REQ_HV, HV_REQ_MISFIT, HV_REQ_QUEUED, HV_REQ_RUNNING, check
from .hv import Problem

__all__ = ["Server", "HV_REQ_HV", "HV_REQ_GRAD", "HV_REQ_MISFIT", "HV_REQ_APPROX"]


class Server:
    def __init__(self, hbm_budget: int, max_concurrent: int = 16, device=None):
        self.lib = _lib.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.hv_server_create(int(hbm_budget), int(max_concurrent), ctypes.byref(h)))
        self._s = h
        self._keep = {}

    def close(self, timeout: float = 600.0):
        if self._s:
            check(self.lib.hv_server_destroy(self._s, float(timeout)))
            self._s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _submit(self, kind, P: Problem | None, m, v=None, k=0, d_obs=None, out=None, phi=None, ckpt=-1, approx=None,
                mode=0):
        r = _lib.HvRequest(kind, P._h if P is not None else None, m.data_ptr() if m is not None else None,
                           v.data_ptr() if v is not None else None, int(k),
                           d_obs.data_ptr() if d_obs is not None else None,
                           out.data_ptr() if out is not None else None,
                           phi.data_ptr() if phi is not None else None, int(ckpt),
                           approx._a if approx is not None else None, int(mode))
        rid = ctypes.c_ulonglong()
        check(self.lib.hv_submit(self._s, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (P, m, v, d_obs, out, phi, approx)
        return rid.value

    def submit_hv(self, P: Problem, m, v, ckpt=-1):
        """Queue H v; returns (request id, output tensor [k, nz, nx])."""
        out = torch.empty(v.shape, dtype=torch.float32, device=self.device)
        return self._submit(HV_REQ_HV, P, m, v=v, k=v.shape[0], out=out, ckpt=ckpt), out

    def submit_grad(self, P: Problem, m, d_obs, ckpt=-1):
        """Queue (phi, grad); returns (request id, phi 0-d float64 tensor, gradient tensor)."""
        phi = torch.empty((), dtype=torch.float64, device=self.device)
        g = torch.empty((P.nz, P.nx), dtype=torch.float32, device=self.device)
        return self._submit(HV_REQ_GRAD, P, m, d_obs=d_obs, out=g, phi=phi, ckpt=ckpt), phi, g

    def submit_approx(self, A, v, mode: int = 0):
        """Queue the apply of a built Hessian approximation to v[k, nz, nx] in an HV_APPROX_* mode
        (hv_approx_apply); returns (request id, output tensor)."""
        out = torch.empty(v.shape, dtype=torch.float32, device=self.device)
        return self._submit(HV_REQ_APPROX, None, None, v=v, k=v.shape[0], out=out, approx=A, mode=mode), out

    def submit_misfit(self, P: Problem, m, d_obs):
        phi = torch.empty((), dtype=torch.float64, device=self.device)
        return self._submit(HV_REQ_MISFIT, P, m, d_obs=d_obs, phi=phi), phi

    def set_batching(self, max_vectors: int) -> None:
        """Merge queued requests on one problem and model into one call of up to max_vectors Born
        vectors (< 2: no merging; hv_server_set_batching)."""
        check(self.lib.hv_server_set_batching(self._s, int(max_vectors)))

    def set_engine(self, slots: int) -> None:
        """Misfit requests join a per-problem lane of up to `slots` models at its next time step (0: misfits run
        as calls; hv_server_set_engine)."""
        check(self.lib.hv_server_set_engine(self._s, int(slots)))

    def set_engine_loop(self, enable: bool) -> None:
        """Misfit lanes created from now on are served by the engine's device-resident loop instead of ticks
        enqueued by the server's thread (hv_server_set_engine_loop)."""
        check(self.lib.hv_server_set_engine_loop(self._s, int(bool(enable))))

    def poll(self, rid: int) -> int:
        st = ctypes.c_int()
        check(self.lib.hv_poll(self._s, int(rid), ctypes.byref(st)))
        return st.value

    def wait(self, rid: int, timeout: float = 600.0) -> int:
        """Block until the request is done; returns its status (0 = HV_OK)."""
        st = ctypes.c_int()
        check(self.lib.hv_wait(self._s, int(rid), float(timeout), ctypes.byref(st)))
        if st.value not in (HV_REQ_QUEUED, HV_REQ_RUNNING):
            self._keep.pop(rid, None)
        return st.value

    def info(self, rid: int) -> dict:
        i = _lib.HvRequestInfo()
        check(self.lib.hv_request_get_info(self._s, int(rid), ctypes.byref(i)))
        return {"kind": i.kind, "status": i.status, "t_submit": i.t_submit, "t_start": i.t_start,
                "t_done": i.t_done, "ws_bytes": i.ws_bytes, "batch": i.batch}
