"""Batched construction workload: H applied to 64 vectors at once (48 impulse
lattices for point-spread functions, paper section 3.2, and 16 Rademacher probes)
over 32 shots on the 64x64 (+20 sponge) model, every time level stored, tile
shapes autotuned, the launch sequence replayed as a CUDA graph."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem
from tests._helpers import f32, oracle_problem, rel

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.fixture(scope="module")
def batched():
    w = synth.workload(3)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v, dtype=torch.float32, device="cuda")
    return w, P, m, v


def test_batched_hessian_parity_on_sampled_vectors(batched, tmp_path):
    w, P, m, v = batched
    P.autotune(k=w.k, cache=str(tmp_path / "tiles.json"))
    P.set_graphs(True)
    Hv = P.hessian_apply(m, v, ckpt=HV_CKPT_ALL)
    Hv2 = P.hessian_apply(m, v, ckpt=HV_CKPT_ALL)            # graph replay
    torch.cuda.synchronize()
    Hv, Hv2 = Hv.cpu().numpy(), Hv2.cpu().numpy()
    assert np.array_equal(Hv, Hv2)
    pick = [0, 23, 47, 48, 63]
    ref = O.hessian_apply(oracle_problem(w), f32(w.m), f32(w.v[pick]))
    for i, j in enumerate(pick):
        assert rel(Hv[j], ref[i]) < TOL, (j, rel(Hv[j], ref[i]))


def test_tile_shapes_and_graphs_do_not_change_results(batched):
    w, P, m, v = batched
    vs = v[[0, 50]].contiguous()
    P.set_graphs(False)
    P.set_tiles((0, 0, 0))
    ref = P.hessian_apply(m, vs, ckpt=7).cpu().numpy()
    for cfg in [(1, 1, 1), (2, 2, 2), (3, 3, 3), (4, 4, 4), (5, 5, 5), (6, 6, 6), (7, 7, 7), (3, 1, 2), (5, 4, 0)]:
        P.set_tiles(cfg)
        for graphs in (False, True):
            P.set_graphs(graphs)
            out = P.hessian_apply(m, vs, ckpt=7).cpu().numpy()
            assert np.array_equal(out, ref), (cfg, graphs)
    P.set_graphs(False)
    P.set_tiles((0, 0, 0))
