"""Misfits at several models in one forward sweep (hv_misfit_models: the
likelihoods of several gpCN chains' proposals, section 2.3): every entry is
bitwise the single-model misfit (hv_misfit) and matches the FP64 oracle's
misfit; ragged shot counts, per-model data, one model, graph replay and the
eager path, and the 64-chain request shape of the serving source."""
import time

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import HV_LAUNCH_DATAFLOW, HV_LAUNCH_PDL, HV_LAUNCH_PLAIN, Problem
from tests._helpers import f32, oracle_problem

pytestmark = pytest.mark.gpu


def make(nz, nx, ns, nt, seed):
    m = synth.gradient_grf_model(seed, nz, nx, 10.0)
    acq = synth.surface_acquisition(nx, ns, nx // 2)
    w = synth.Workload(name=f"{nz}x{nx}", nz=nz, nx=nx, nb=20, h=10.0, nt=nt, dt=synth.cfl_dt(10.0, float(m.max())),
                       f0=15.0, t0=0.1, vmax=float(m.max()), acq=acq, m=m,
                       v=synth.smoothed_normal_vectors(seed + 1, 1, nz, nx))
    return w, Problem.from_workload(w)


def proposals(w, k, seed, amp=0.03):
    """k smooth perturbations of the model, capped at the velocity the time step was chosen for."""
    z = synth.smoothed_normal_vectors(seed, k, w.nz, w.nx, 4.0)
    z /= np.abs(z).max(axis=(1, 2), keepdims=True)
    return np.minimum(w.m[None] * (1.0 + amp * z), w.vmax).astype(np.float32)


def t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def ragged():
    w, P = make(48, 64, 11, 300, 31)             # 11 shots: one full group of 8 and a ragged one of 3
    dobs = O.fwd_model(oracle_problem(w), f32(w.m), nthreads=8)
    return w, P, dobs


def test_models_bitwise_single_and_match_the_oracle(ragged):
    w, P, dobs = ragged
    ms = proposals(w, 5, 41)
    phi = P.misfit_models(t(ms), t(dobs)).cpu().numpy()
    single = np.array([float(P.misfit(t(ms[i]), t(dobs))) for i in range(5)])
    assert np.array_equal(phi, single), (phi, single)
    for i in (0, 3):
        ref = O.misfit_grad(oracle_problem(w), f32(ms[i]), f32(dobs), nthreads=8)[0]
        assert abs(phi[i] - ref) < 2e-4 * ref, (i, phi[i], ref)
    assert len(set(phi.tolist())) == 5          # the models differ, so do their misfits


def test_per_model_data(ragged):
    w, P, dobs = ragged
    ms = proposals(w, 3, 43)
    noise = synth.normal(47, 3 * dobs.size).reshape((3,) + dobs.shape) * 1e-3
    D = (dobs[None] + noise).astype(np.float32)
    phi = P.misfit_models(t(ms), t(D)).cpu().numpy()
    for i in range(3):
        assert phi[i] == float(P.misfit(t(ms[i]), t(D[i]))), i


def test_one_model_graphs_and_launch_modes(ragged):
    w, P, dobs = ragged
    ms = proposals(w, 2, 53)
    one = float(P.misfit(t(ms[:1][0]), t(dobs)))
    assert float(P.misfit_models(t(ms[:1]), t(dobs))[0]) == one
    first = P.misfit_models(t(ms), t(dobs)).cpu().numpy()       # eager launches
    try:
        P.set_graphs(True)
        for _ in range(2):                                         # captured, then replayed
            assert np.array_equal(P.misfit_models(t(ms), t(dobs)).cpu().numpy(), first)
        P.set_graphs(False)
        for mode in (HV_LAUNCH_PLAIN, HV_LAUNCH_DATAFLOW, HV_LAUNCH_PDL):
            P.set_launch_mode(mode)
            assert np.array_equal(P.misfit_models(t(ms), t(dobs)).cpu().numpy(), first), mode
    finally:
        P.set_graphs(False)
        P.set_launch_mode(HV_LAUNCH_PDL)


def test_chain_request_shape_64_models():
    """The serving source's chains: 64 proposals on a 128 x 128, 8-shot, 1000-step problem."""
    w, P = make(128, 128, 8, 1000, 61)
    ms = t(proposals(w, 64, 67))
    dobs = t(synth.normal(71, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr) * 1e-3)
    phi = P.misfit_models(ms, dobs)
    torch.cuda.synchronize()
    for i in (0, 17, 63):
        assert float(phi[i]) == float(P.misfit(ms[i], dobs)), i
    for _ in range(2):
        P.misfit_models(ms, dobs)
        P.misfit(ms[0], dobs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.misfit_models(ms, dobs)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for i in range(8):
        P.misfit(ms[i], dobs)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    print(f"64 misfits in one sweep: {64 / (t1 - t0):.0f}/s; one at a time: {8 / (t2 - t1):.0f}/s")
