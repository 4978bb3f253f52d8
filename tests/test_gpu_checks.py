"""Output checks: the non-finite scan (hv_count_nonfinite) counts exactly the
NaN and +-Inf entries planted (on the host) in an array of ragged length, sees
none in an empty one, and none in the H v of a stable run."""
import numpy as np
import pytest
import torch

from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import Problem, count_nonfinite

pytestmark = pytest.mark.gpu


def test_counts_planted_nonfinite_values():
    n = 1_000_003
    x = synth.normal(301, n).astype(np.float32)
    pos = (synth.uniform(303, 25) * n).astype(np.int64)
    pos = np.unique(pos)
    kinds = [np.nan, np.inf, -np.inf]
    for i, p in enumerate(pos):
        x[p] = kinds[i % 3]
    assert count_nonfinite(torch.tensor(x, device="cuda")) == len(pos)
    assert count_nonfinite(torch.tensor(x[:0], device="cuda")) == 0
    x[pos] = 1.0
    assert count_nonfinite(torch.tensor(x, device="cuda")) == 0


def test_a_stable_hessian_apply_is_finite():
    w = synth.workload(1, nt=200)
    P = Problem.from_workload(w)
    Hv = P.hessian_apply(torch.tensor(w.m, dtype=torch.float32, device="cuda"),
                         torch.tensor(w.v, dtype=torch.float32, device="cuda"), ckpt=5)
    assert count_nonfinite(Hv.contiguous()) == 0
