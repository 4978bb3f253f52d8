"""The allocation-free Hessian apply (hv_hessian_apply_static).

Some callers cannot allocate device memory where they call the library: an
application that hands out all device memory from its own pool, or a
real-time loop that must not stall in an allocator.  For them the library
keeps one fixed scratch array per GPU and offers a Hessian apply that needs
neither a handle nor a workspace.  These checks call it through the C ABI:
two calls in a row must equal the workspace-based hv_hessian_apply with the
same tile configuration bitwise (same kernels, same order of operations) and
the FP64 oracle within the accuracy bar; a following call of another shape
must not pick up the previous call's tables; the status word reads HV_OK.
This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import _lib, synth
from paper_2507_10804_gb300.hv import Problem
from tests._helpers import f32, oracle_problem, ragged_workload, rel

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


def _static_status(lib):
    st = ctypes.c_int(-1)
    _lib.check(lib.hv_static_status(ctypes.byref(st)))
    return st.value


def _workspace_version(w, m, v, ckpt):
    P = Problem.from_workload(w)
    P.set_tiles([0, 0, 0])                      # the static path runs tile configuration 0
    out = P.hessian_apply(m, v, ckpt=ckpt)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_scratch_hessian_apply_matches_workspace_version():
    lib = _lib.load()
    w = synth.workload(3, nt=300, ns=2)                       # 64x64 + 20-cell sponge, 2 shots
    w.v = w.v[[0, 50]]                                        # one impulse lattice, one Rademacher vector
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    ref_h = _workspace_version(w, m, v, 12)
    oracle = O.hessian_apply(oracle_problem(w), f32(w.m), f32(w.v), nthreads=2)
    g, a, keep = _structs(w)
    out = torch.empty_like(v)
    for call in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call(lib, g, a, m, v, out, 12)
        torch.cuda.synchronize()
        _lib.check(rc)
        free_after = torch.cuda.mem_get_info()[0]
        got = out.cpu().numpy()
        assert np.array_equal(got, ref_h), call
        for j in range(v.shape[0]):
            assert rel(got[j], oracle[j]) < TOL, (call, j)
        if call == 1:                                        # set-up done: nothing more is allocated
            assert free_after >= free_before - (2 << 20)
    assert _static_status(lib) == _lib.HV_OK

    # Another shape right after: fewer shots and receivers, another grid and budget.
    w2 = ragged_workload(nz=29, nx=53, nb=5, nt=90, ns=1, nr=5, k=2)
    m2 = torch.tensor(w2.m, dtype=torch.float32, device="cuda")
    v2 = torch.tensor(w2.v, dtype=torch.float32, device="cuda")
    ref2 = _workspace_version(w2, m2, v2, 4)
    g2, a2, keep2 = _structs(w2)
    out2 = torch.full_like(v2, float("nan"))
    _lib.check(_call(lib, g2, a2, m2, v2, out2, 4))
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy(), ref2)
    assert _static_status(lib) == _lib.HV_OK


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


def test_static_scratch_refuses_stream_capture():
    lib = _lib.load()
    w = ragged_workload(nt=20, ns=1, k=1)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    out = torch.empty_like(v)
    g, a, keep = _structs(w)
    _lib.check(_call(lib, g, a, m, v, out, 3))               # set-up outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.stream(s):
        graph.capture_begin()
        try:
            rc = _call(lib, g, a, m, v, out, 3)
        finally:
            graph.capture_end()
    assert rc == _lib.HV_EINVAL
    assert "captured" in lib.hv_last_error().decode()
