"""The Hessian apply split over shot blocks (section 3: H_d v is a sum over
sources; eq. (grad) sums the imaging over sources), on one GPU: each block's
extended image (hv_hessian_apply_partial) against the FP64 oracle's, and the
blocks' images summed in order and folded once (hv_image_fold) against the
whole apply."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import Problem
from paper_2507_10804_gb300.parallel import shard_problem, sharded_hessian_apply
from tests._helpers import f32, oracle_problem, ragged_workload, rel

pytestmark = pytest.mark.gpu
TOL = 2e-4


def test_partial_image_matches_oracle_and_folds_to_the_apply():
    w = ragged_workload(nt=120, ns=3, k=2)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    ext = P.hessian_apply_partial(m, v, ckpt=6)
    Hv = P.hessian_apply(m, v, ckpt=6, out_dtype=torch.float64)
    folded = P.fold(ext, out_dtype=torch.float64)
    folded32 = P.fold(ext)
    torch.cuda.synchronize()
    ext, Hv, folded, folded32 = (t.cpu().numpy() for t in (ext, Hv, folded, folded32))
    ref = O.hessian_image(oracle_problem(w), f32(w.m), f32(w.v), nthreads=3)
    for j in range(2):
        assert rel(ext[j], ref[j]) < TOL, j
        assert rel(folded[j], Hv[j]) < 1e-12, j          # fold order only: FP64 rounding
    assert np.array_equal(folded32, folded.astype(np.float32))


def test_two_shot_blocks_sum_to_the_whole_apply():
    """16 shots as two blocks of 8 (the shot groups of the whole apply), images summed in block order."""
    w = synth.workload(3, nt=200, ns=16)
    w.v = w.v[[3, 49]]
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    full = Problem.from_workload(w).hessian_apply(m, v, ckpt=10, out_dtype=torch.float64)
    blocks = [shard_problem(Problem, w, r, 2) for r in range(2)]
    exts = [B.hessian_apply_partial(m, v, ckpt=10) for B in blocks]
    split = sharded_hessian_apply(lambda: exts[0] + exts[1], lambda e: blocks[0].fold(e, torch.float64))
    torch.cuda.synchronize()
    full, split = full.cpu().numpy(), split.cpu().numpy()
    for j in range(2):
        assert rel(split[j], full[j]) < 1e-12, j
