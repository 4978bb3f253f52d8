"""Shared-memory-resident H v (hv_set_resident) against the FP64 oracle and the
tiled path: the same H v to rounding (only the image's summation order
differs), bitwise independent of k and of graph replay, and the tiled path
where the grid does not fit."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem
from tests._helpers import f32, oracle_problem, ragged_workload, rel

pytestmark = pytest.mark.gpu
TOL = 2e-4


def gpu(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _dense_receivers(w):
    """Receivers on every node of two rows (several per thread block, both rows of a block)."""
    nx, ns = w.nx, w.ns
    rec_ix = np.tile(np.r_[np.arange(nx), np.arange(nx)], ns).astype(np.int32)
    rec_iz = np.tile(np.r_[np.full(nx, 2), np.full(nx, 3)], ns).astype(np.int32)
    acq = synth.Acquisition(src_iz=w.acq.src_iz, src_ix=w.acq.src_ix, rec_iz=rec_iz.reshape(ns, -1),
                            rec_ix=rec_ix.reshape(ns, -1))
    return synth.Workload(name=w.name, nz=w.nz, nx=w.nx, nb=w.nb, h=w.h, nt=w.nt, dt=w.dt, f0=w.f0, t0=w.t0,
                          vmax=w.vmax, acq=acq, m=w.m, v=w.v, sigma=w.sigma)


CASES = {
    "cfg1": lambda: synth.workload(1),
    # padded 49 x 84: an odd row count (the last thread block is half outside)
    "ragged": lambda: ragged_workload(nz=37, nx=72, nb=6, nt=150, ns=3, nr=7, k=3),
    "dense_receivers": lambda: _dense_receivers(ragged_workload(nz=30, nx=60, nb=6, nt=120, ns=2, nr=4, k=2)),
    # padded 100 x 116: 1450 thread blocks, more than three per thread (the four-block kernels), and shared
    # memory near the per-CTA limit
    "four_blocks": lambda: ragged_workload(nz=88, nx=104, nb=6, nt=60, ns=2, nr=5, k=2),
}


@pytest.mark.parametrize("case", list(CASES))
def test_resident_matches_oracle_and_tiled_path(case):
    w = CASES[case]()
    P = Problem.from_workload(w)
    m, v = gpu(w.m), gpu(w.v)
    tiled = host(P.hessian_apply(m, v, ckpt=HV_CKPT_ALL))
    assert P.set_resident(True)
    res = host(P.hessian_apply(m, v, ckpt=HV_CKPT_ALL))
    for j in range(v.shape[0]):
        assert rel(res[j], tiled[j]) < 2e-6, (case, j, rel(res[j], tiled[j]))
    want = O.hessian_apply(oracle_problem(w), f32(w.m), f32(w.v))
    for j in range(v.shape[0]):
        assert rel(res[j], want[j]) < TOL, (case, j, rel(res[j], want[j]))
    # a checkpointed call still takes the tiled path
    assert np.array_equal(host(P.hessian_apply(m, v, ckpt=5)), host(P.hessian_apply(m, v, ckpt=7)))
    assert P.status() == 0


def test_resident_is_bitwise_independent_of_k_and_graphs():
    w = ragged_workload(nz=37, nx=72, nb=6, nt=120, ns=3, nr=7, k=5)
    P = Problem.from_workload(w)
    assert P.set_resident(True)
    m, v = gpu(w.m), gpu(w.v)
    P.set_graphs(False)
    batch = host(P.hessian_apply(m, v))
    P.set_graphs(True)
    assert np.array_equal(host(P.hessian_apply(m, v)), batch)
    for j in (0, 3):
        assert np.array_equal(host(P.hessian_apply(m, v[j:j + 1].contiguous()))[0], batch[j]), j


def test_grid_that_does_not_fit_takes_the_tiled_path():
    w = ragged_workload(nz=37, nx=71, nb=6, nt=100, ns=2, nr=5, k=2)     # padded width 83: not a multiple of 4
    P = Problem.from_workload(w)
    m, v = gpu(w.m), gpu(w.v)
    ref = host(P.hessian_apply(m, v))
    assert not P.set_resident(True)
    assert np.array_equal(host(P.hessian_apply(m, v)), ref)
