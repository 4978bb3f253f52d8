"""The 384 x 1152 (+40 sponge) workload's Hessian apply against the FP64 oracle.

Paper section 3 (opening): H_d v = F* Gamma^-1 F v costs two wave solves per
source, the forward field a third; eq. (grad) sums the imaging over sources.
The GPU runs the benchmark's launch configuration: the full padded grid
(464 x 1232), the tile shapes the autotuner picks for the 32-shot problem,
30 snapshots per shot with binomial recomputation, and shot groups of up to
8 shots (two groups here, 5 + 4 shots, so the group sums meet the oracle too).
The oracle keeps every time level, so the shot subset and the step count are
kept modest (9 shots, 400 steps: about 6 G point updates on the host).

The imaging sum is checked separately on the whole workload (32 shots,
3000 steps): the default per-step FP32 group sums added to double-float images
against every shot's product added in FP64.
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300._lib import HV_IMAGE_FP64, HV_IMAGE_PAIRS
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem
from tests._helpers import f32, oracle_problem, rel

pytestmark = pytest.mark.gpu
TOL = 2e-4
SHOTS = [0, 4, 8, 12, 16, 19, 23, 27, 31]     # 9 of the 32 shots: groups of 5 and 4


def _subset(w, shots, nt):
    ws = synth.workload(2, nt=nt)
    a = w.acq
    ws.acq = synth.Acquisition(a.src_iz[shots], a.src_ix[shots], a.rec_iz[shots], a.rec_ix[shots])
    return ws


@pytest.fixture(scope="module")
def bench_tiles():
    """The tiles the benchmark runs: autotuned on the 32-shot, one-vector problem."""
    w = synth.workload(2, nt=50)
    P = Problem.from_workload(w)
    tiles = P.autotune(k=1)
    P.close()
    return tiles


def test_fullsize_hessian_apply_matches_oracle(bench_tiles):
    w = synth.workload(2)
    ws = _subset(w, SHOTS, 400)
    P = Problem.from_workload(ws)
    P.set_tiles(bench_tiles)
    vv = synth.smoothed_normal_vectors(5150, 2, w.nz, w.nx, 3.0)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(vv, dtype=torch.float32, device="cuda")
    H30 = P.hessian_apply(m, v, ckpt=30)
    Hall = P.hessian_apply(m, v, ckpt=HV_CKPT_ALL)
    torch.cuda.synchronize()
    assert P.status() == 0
    H30, Hall = H30.cpu().numpy(), Hall.cpu().numpy()
    assert np.array_equal(H30, Hall)                 # recomputation from 30 snapshots is bitwise neutral
    nthreads = max(1, min(len(SHOTS), (os.cpu_count() or 1) // 2))
    ref = O.hessian_apply(oracle_problem(ws), f32(w.m), f32(vv), nthreads=nthreads)
    for j in range(2):
        err = rel(H30[j], ref[j])
        assert err < TOL, (j, err)


def test_fullsize_image_sum_against_fp64_accumulation(bench_tiles):
    """32 shots x 3000 steps, 30 snapshots: the default imaging sum against exact products summed in FP64."""
    w = synth.workload(2)
    P = Problem.from_workload(w)
    P.set_tiles(bench_tiles)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    H = P.hessian_apply(m, v, ckpt=30, out_dtype=torch.float64)
    P.set_image_precision(HV_IMAGE_FP64)
    H64 = P.hessian_apply(m, v, ckpt=30, out_dtype=torch.float64)
    P.set_image_precision(HV_IMAGE_PAIRS)
    again = P.hessian_apply(m, v, ckpt=30, out_dtype=torch.float64)
    torch.cuda.synchronize()
    assert P.status() == 0
    H, H64, again = H.cpu().numpy(), H64.cpu().numpy(), again.cpu().numpy()
    assert np.array_equal(H, again)
    d = rel(H, H64)
    dmax = float(np.max(np.abs(H - H64)) / np.max(np.abs(H64)))
    print(f"imaging sum, default vs FP64 accumulation: rel L2 {d:.3e}, max abs / max {dmax:.3e}")
    assert d < 1e-5, d                                 # a small fraction of the 2e-4 budget
