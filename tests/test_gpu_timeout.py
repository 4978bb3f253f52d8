"""Failure detection on the device without a fault: a bounded wait that runs out.

In the dataflow launch mode every CTA waits, before it issues any bulk copy,
until the tiles it reads have been finished by the earlier steps (per-tile
counters).  hv_inject_wait_timeout makes one step wait for a count that no
step reaches -- a flag nothing sets -- with a short wait limit.  The kernels
must give up, report HV_ETIMEOUT through hv_status and leave the context and
the handle usable: the next call is clean and bitwise the same as before.
"""
import time

import numpy as np
import pytest
import torch

from paper_2507_10804_gb300._lib import HV_ETIMEOUT, HV_LAUNCH_DATAFLOW, HV_LAUNCH_PDL, HV_OK
from paper_2507_10804_gb300.hv import Problem
from tests._helpers import ragged_workload

pytestmark = pytest.mark.gpu


def test_dataflow_wait_runs_out_and_the_handle_recovers():
    w = ragged_workload(nt=60)
    P = Problem.from_workload(w)
    P.set_tiles([0, 0, 0])                       # one tiling: the dataflow ordering applies
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    ref = P.hessian_apply(m, v, ckpt=5).cpu().numpy()
    assert P.status() == HV_OK
    P.set_launch_mode(HV_LAUNCH_DATAFLOW)
    flow = P.hessian_apply(m, v, ckpt=5).cpu().numpy()
    assert P.status() == HV_OK
    assert np.array_equal(flow, ref)

    P.set_wait_limit(0.005)
    P.inject_wait_timeout()
    t0 = time.perf_counter()
    P.hessian_apply(m, v, ckpt=5)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert P.status() == HV_ETIMEOUT
    assert elapsed < 10.0                        # every later wait gave up at once
    assert P.status() == HV_OK                   # reading the status cleared it

    P.set_wait_limit(2.0)
    again = P.hessian_apply(m, v, ckpt=5).cpu().numpy()
    assert P.status() == HV_OK
    assert np.array_equal(again, ref)
    P.set_launch_mode(HV_LAUNCH_PDL)
    assert np.array_equal(P.hessian_apply(m, v, ckpt=5).cpu().numpy(), ref)
    assert P.status() == HV_OK


def test_wait_limit_is_validated():
    w = ragged_workload(nt=10)
    P = Problem.from_workload(w)
    from paper_2507_10804_gb300._lib import HvError
    for bad in (0.0, -1.0, 1e-6, 120.0):
        with pytest.raises(HvError):
            P.set_wait_limit(bad)
    P.set_wait_limit(1.0)
