"""Batched construction workload: H applied to 64 vectors at once (48 impulse
lattices for point-spread functions, paper section 3.2, and 16 Rademacher probes)
over 32 shots on the 64x64 (+20 sponge) model, every time level stored, tile
shapes autotuned, the launch sequence replayed as a CUDA graph."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import (HV_CKPT_ALL, HV_LAUNCH_DATAFLOW, HV_LAUNCH_PDL, HV_LAUNCH_PLAIN, Problem,
                                       menu_size)
from tests._helpers import f32, oracle_problem, ragged_workload, rel

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
    n = menu_size()
    cfgs = [(c, c, c) for c in range(1, n)] + [(3, 1, 2), (5, 4, 0), (9, 12, 13), (15, 8, 10)]
    for cfg in cfgs:
        P.set_tiles(cfg)
        for graphs in (False, True):
            P.set_graphs(graphs)
            out = P.hessian_apply(m, vs, ckpt=7).cpu().numpy()
            assert np.array_equal(out, ref), (cfg, graphs)
    for mode in (HV_LAUNCH_PLAIN, HV_LAUNCH_PDL, HV_LAUNCH_DATAFLOW):
        P.set_launch_mode(mode)
        for graphs in (False, True):
            P.set_graphs(graphs)
            out = P.hessian_apply(m, vs, ckpt=7).cpu().numpy()
            assert np.array_equal(out, ref), (mode, graphs)
    P.set_graphs(False)
    P.set_tiles((0, 0, 0))


def test_shot_groups_spanning_ctas_ragged_shot_count():
    """20 shots form adjoint groups of 7, 7 and 6; configurations that walk two or
    four groups per CTA, or keep two shots in flight, give bitwise the same H v."""
    w = ragged_workload(nt=120, ns=20, nr=9, k=2)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v[:2], dtype=torch.float32, device="cuda")
    P.set_tiles((0, 0, 0))
    ref = P.hessian_apply(m, v, ckpt=5).cpu().numpy()
    for c in range(1, menu_size()):
        P.set_tiles((c, c, c))
        out = P.hessian_apply(m, v, ckpt=5).cpu().numpy()
        assert np.array_equal(out, ref), c
    want = O.hessian_apply(oracle_problem(w), f32(w.m), f32(w.v[:2]))
    for j in range(2):
        assert rel(ref[j], want[j]) < TOL, (j, rel(ref[j], want[j]))


@pytest.mark.parametrize("tiles", [(6, 8, 6), (9, 10, 9), (7, 11, 13)])
def test_dataflow_launch_mode_bitwise(tiles):
    """Steps that start on tile-neighbourhood counters give the same bits as
    fully serialised steps: H v (binomial and stored history, k = 3 with Born
    items per vector), the gradient (a residual kernel between the sweeps) and
    the Born map, on a ragged grid with 20 shots (groups of 7, 7, 6)."""
    w = ragged_workload(nt=90, ns=20, nr=9, k=3)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v[:3], dtype=torch.float32, device="cuda")
    dobs = torch.tensor(O.fwd_model(oracle_problem(w), f32(w.m) * 1.01), dtype=torch.float32, device="cuda")
    P.set_tiles(tiles)

    def run():
        out = [P.hessian_apply(m, v, ckpt=4), P.hessian_apply(m, v, ckpt=HV_CKPT_ALL), P.born(m, v)]
        phi, g = P.misfit_grad(m, dobs, ckpt=6)
        out += [g, phi.reshape(1)]
        torch.cuda.synchronize()
        return [x.cpu().numpy() for x in out]

    P.set_launch_mode(HV_LAUNCH_PLAIN)
    ref = run()
    for mode in (HV_LAUNCH_DATAFLOW, HV_LAUNCH_PDL, HV_LAUNCH_DATAFLOW):
        P.set_launch_mode(mode)
        got = run()
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), mode
    assert P.status() == 0


@pytest.mark.parametrize("tiles", [(0, 0, 0), (2, 6, 5), (4, 5, 7), (3, 3, 3), (9, 10, 13), (1, 15, 1)])
def test_fused_double_steps_bitwise_equal_single_steps(tiles):
    """The recomputation's fused double steps (u^n with an 8-cell halo, the extended
    ring recomputed and zeroed off the padded grid) give the same bits as single steps:
    H v with k = 2 and the gradient, binomial schedules with many recomputed steps, on a
    ragged grid whose tiles and rings cross all four edges."""
    w = ragged_workload(nt=140, ns=5, nr=6, k=2)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(w.v[:2], dtype=torch.float32, device="cuda")
    dobs = torch.tensor(O.fwd_model(oracle_problem(w), f32(w.m) * 1.01), dtype=torch.float32, device="cuda")
    P.set_tiles(tiles)

    def run():
        out = [P.hessian_apply(m, v, ckpt=3), P.hessian_apply(m, v, ckpt=9)]
        phi, g = P.misfit_grad(m, dobs, ckpt=4)
        out += [g, phi.reshape(1)]
        torch.cuda.synchronize()
        return [x.cpu().numpy() for x in out]

    P.set_step_fusion(False)
    ref = run()
    P.set_step_fusion(True)
    for graphs in (False, True):
        P.set_graphs(graphs)
        for a, b in zip(run(), ref):
            assert np.array_equal(a, b), (tiles, graphs)
    assert P.status() == 0
