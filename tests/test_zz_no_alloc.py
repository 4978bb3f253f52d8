"""The allocation-free Hessian apply (hv_hessian_apply_static).

Some callers cannot allocate device memory where they call the library: an
application that hands out all device memory from its own pool, or a
real-time loop that must not stall in an allocator.  For them the library
keeps one fixed scratch array per GPU and offers a Hessian apply that needs
neither a handle nor a workspace.  These checks call it through the C ABI and
compare it with the workspace-based hv_hessian_apply on two calls in a row.
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2507_10804_gb300 import _lib, synth
from paper_2507_10804_gb300.hv import Problem
from tests._helpers import rel

pytestmark = pytest.mark.gpu
TOL = 2e-4


def _structs(w):
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))
            for a in (w.acq.src_iz, w.acq.src_ix, w.acq.rec_iz, w.acq.rec_ix)]
    g = _lib.HvGrid(w.nz, w.nx, w.nb, w.h)
    a = _lib.HvAcq(w.ns, arrs[0].ctypes.data_as(_lib.ip), arrs[1].ctypes.data_as(_lib.ip), w.nr,
                   arrs[2].ctypes.data_as(_lib.ip), arrs[3].ctypes.data_as(_lib.ip), w.nt, w.dt, w.f0, w.t0,
                   w.vmax, w.R, w.sigma)
    return g, a, arrs


def _call(lib, g, a, m, v, out, ckpt):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.hv_hessian_apply_static(ctypes.byref(g), ctypes.byref(a), m.data_ptr(), v.data_ptr(), v.shape[0],
                                       out.data_ptr(), ckpt, stream)


def test_static_scratch_hessian_apply_matches_workspace_version():
    lib = _lib.load()
    w = synth.workload(3, nt=300, ns=2)                       # 64x64 + 20-cell sponge, 2 shots
    w.v = w.v[[0, 50]]                                        # one impulse lattice, one Rademacher vector
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    ref = Problem.from_workload(w).hessian_apply(m, v, ckpt=12)
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    g, a, keep = _structs(w)
    out = torch.empty_like(ref)
    for call in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call(lib, g, a, m, v, out, 12)
        torch.cuda.synchronize()
        _lib.check(rc)
        free_after = torch.cuda.mem_get_info()[0]
        got = out.cpu().numpy()
        for j in range(v.shape[0]):
            assert rel(got[j], ref_h[j]) < TOL, (call, j)
        if call == 1:                                        # set-up done: nothing more is allocated
            assert free_after >= free_before - (2 << 20)


def test_static_scratch_rejects_problems_beyond_its_size():
    lib = _lib.load()
    w = synth.workload(2, nt=50, ns=2)                        # 464x1232 padded: far beyond 64 MiB
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    out = torch.empty_like(v)
    g, a, keep = _structs(w)
    rc = _call(lib, g, a, m, v, out, 4)
    assert rc == _lib.HV_ENOMEM
    assert "static array holds" in lib.hv_last_error().decode()
