"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar (from the method's accuracy target): relative L2 error <= 2e-4 on
wavefields, data, gradients and Hessian applies; source and receiver indexing
bit-exact; checkpointed and stored-history adjoints bitwise identical.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem
from tests._helpers import f32, oracle_problem, ragged_workload, rel

pytestmark = pytest.mark.gpu
TOL = 2e-4


def gpu(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def cfg1():
    w = synth.workload(1)
    return w, Problem.from_workload(w), oracle_problem(w)


@pytest.fixture(scope="module")
def ragged():
    w = ragged_workload()
    return w, Problem.from_workload(w), oracle_problem(w)


# ------------------------------------------------------------------ indexing
def test_source_and_receiver_indexing_bit_exact():
    """One step from rest: u^1 = C s_0 / (1 + a) at the source node only.  Two steps:
    every receiver sample equals the wavefield at its node bitwise."""
    w = ragged_workload(nt=2, ns=4, nr=9)
    w.t0 = 0.0                      # s(0) = 1
    P = Problem.from_workload(w)
    m = gpu(w.m)
    U = host(P.wavefield(m, [0, 1]))                     # [2, ns, NZ, NX]
    for s in range(w.ns):
        nz_idx = np.argwhere(U[0, s] != 0.0)
        assert nz_idx.tolist() == [[w.acq.src_iz[s] + w.nb, w.acq.src_ix[s] + w.nb]]
    d = host(P.fwd_model(m))                             # d[s, n, r] = u^{n+1}[rec]
    for s in range(w.ns):
        for r in range(w.nr):
            z, x = w.acq.rec_iz[s, r] + w.nb, w.acq.rec_ix[s, r] + w.nb
            assert d[s, 1, r] == U[1, s, z, x]
            assert d[s, 0, r] == U[0, s, z, x]
    # and the same nodes are nonzero in the oracle's data
    Or = O.fwd_model(oracle_problem(w), f32(w.m))
    assert np.array_equal(d[:, 1] != 0.0, Or[:, 1] != 0.0)


# ------------------------------------------------------------------ forward
def test_wavefield_parity_cfg1(cfg1):
    w, P, OP = cfg1
    steps = [99, 299, 599]
    U = host(P.wavefield(gpu(w.m), steps))[:, 0]
    Uo = O.wavefield(OP, f32(w.m), 0)[steps]
    for i in range(len(steps)):
        assert rel(U[i], Uo[i]) < TOL, (steps[i], rel(U[i], Uo[i]))


def test_fwd_model_parity_cfg1(cfg1):
    w, P, OP = cfg1
    d = host(P.fwd_model(gpu(w.m)))
    assert rel(d, O.fwd_model(OP, f32(w.m))) < TOL


def test_fwd_model_parity_ragged_multishot(ragged):
    w, P, OP = ragged
    d = host(P.fwd_model(gpu(w.m)))
    assert rel(d, O.fwd_model(OP, f32(w.m))) < TOL


def test_born_parity_ragged_multivector(ragged):
    w, P, OP = ragged
    dd = host(P.born(gpu(w.m), gpu(w.v)))
    ref = O.born(OP, f32(w.m), f32(w.v))
    for j in range(w.k):
        assert rel(dd[j], ref[j]) < TOL


def test_migrate_parity_ragged(ragged):
    w, P, OP = ragged
    r = synth.normal(77, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr)
    g = host(P.migrate(gpu(w.m), gpu(r)))
    assert rel(g, O.adjoint(OP, f32(w.m), f32(r))) < TOL


def test_misfit_grad_parity_ragged(ragged):
    w, P, OP = ragged
    dobs = O.fwd_model(OP, synth.perturbed_model(w.m, w.h, 3, amp=0.05, radius=80.0))
    phi, g = P.misfit_grad(gpu(w.m), gpu(dobs), ckpt=4)
    phi_o, g_o = O.misfit_grad(OP, f32(w.m), f32(dobs))
    assert abs(float(phi) - phi_o) < TOL * phi_o
    assert rel(host(g), g_o) < TOL


# ------------------------------------------------------------------ Hessian
def test_hessian_apply_parity_cfg1(cfg1):
    w, P, OP = cfg1
    Hv = host(P.hessian_apply(gpu(w.m), gpu(w.v)))
    assert rel(Hv, O.hessian_apply(OP, f32(w.m), f32(w.v))) < TOL


def test_hessian_apply_checkpointed_bitwise_equals_history(cfg1):
    w, P, _ = cfg1
    m, v = gpu(w.m), gpu(w.v)
    ref = host(P.hessian_apply(m, v, ckpt=HV_CKPT_ALL))
    for budget in (1, 7, 30):
        assert np.array_equal(host(P.hessian_apply(m, v, ckpt=budget)), ref), budget


def test_hessian_apply_parity_ragged_multivector_and_batching(ragged):
    w, P, OP = ragged
    m, v = gpu(w.m), gpu(w.v)
    Hv = host(P.hessian_apply(m, v, ckpt=5))
    ref = O.hessian_apply(OP, f32(w.m), f32(w.v))
    for j in range(w.k):
        assert rel(Hv[j], ref[j]) < TOL
        alone = host(P.hessian_apply(m, v[j:j + 1].contiguous(), ckpt=5))[0]
        assert np.array_equal(alone, Hv[j])              # same result alone and in the batch
    H64 = host(P.hessian_apply(m, v, ckpt=5, out_dtype=torch.float64))
    assert np.array_equal(H64.astype(np.float32), Hv.astype(np.float32))


def test_hessian_apply_deterministic(ragged):
    w, P, _ = ragged
    m, v = gpu(w.m), gpu(w.v)
    a = host(P.hessian_apply(m, v, ckpt=3))
    b = host(P.hessian_apply(m, v, ckpt=3))
    assert np.array_equal(a, b)


def test_gpu_adjoint_and_symmetry_identities(ragged):
    w, P, _ = ragged
    m = gpu(w.m)
    dm = synth.smoothed_normal_vectors(91, 2, w.nz, w.nx, 1.5)
    r = synth.normal(92, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr)
    Jdm = host(P.born(m, gpu(dm[:1])))[0]
    JTr = host(P.migrate(m, gpu(r)))
    a, b = np.vdot(Jdm, r), np.vdot(f32(dm[0]), JTr)
    assert abs(a - b) < 1e-4 * abs(a)
    H = host(P.hessian_apply(m, gpu(dm), out_dtype=torch.float64))
    u, v = f32(dm[0]), f32(dm[1])
    assert abs(np.vdot(u, H[1]) - np.vdot(H[0], v)) < 1e-4 * abs(np.vdot(u, H[1]))
    assert np.vdot(u, H[0]) > 0


# ------------------------------------------------------------------ degenerate cases
@pytest.mark.parametrize("nz,nx,nb", [(1, 1, 3), (5, 3, 0), (2, 9, 1)])
def test_degenerate_grids(nz, nx, nb):
    w = ragged_workload(nz=nz, nx=nx, nb=nb, nt=40, ns=1, nr=1, k=1)
    w.acq = synth.surface_acquisition(nx, 1, 1, 0, 0)
    P, OP = Problem.from_workload(w), oracle_problem(w)
    m, v = gpu(w.m), gpu(w.v)
    assert rel(host(P.fwd_model(m)), O.fwd_model(OP, f32(w.m))) < TOL
    assert rel(host(P.hessian_apply(m, v, ckpt=2)), O.hessian_apply(OP, f32(w.m), f32(w.v))) < TOL


def test_invalid_calls_raise(ragged):
    w, P, _ = ragged
    from paper_2507_10804_gb300._lib import HvError
    with pytest.raises(HvError):
        P.hessian_apply(gpu(w.m), gpu(w.v), ckpt=0)
    with pytest.raises(ValueError):
        P.hessian_apply(gpu(w.m[:-1]), gpu(w.v))


# ------------------------------------------------------------------ full size
def test_full_size_data_parity_on_sampled_shots():
    """384 x 1152 (+40 sponge), 32 shots, 384 receivers, in the benchmark's launch
    configuration; the oracle recomputes two of the 32 shots (first 400 steps)."""
    w = synth.workload(2, nt=400)
    P = Problem.from_workload(w)
    d = host(P.fwd_model(gpu(w.m)))
    for s in (0, 19):
        ws_ = synth.workload(2, nt=400)
        ws_.acq = synth.Acquisition(w.acq.src_iz[s:s + 1], w.acq.src_ix[s:s + 1], w.acq.rec_iz[s:s + 1],
                                    w.acq.rec_ix[s:s + 1])
        ref = O.fwd_model(oracle_problem(ws_), f32(w.m), nthreads=1)[0]
        assert rel(d[s], ref) < TOL, (s, rel(d[s], ref))


def test_full_size_hessian_symmetry_with_30_snapshots():
    w = synth.workload(2)
    P = Problem.from_workload(w)
    m = gpu(w.m)
    vv = synth.smoothed_normal_vectors(5150, 2, w.nz, w.nx, 3.0)
    H = host(P.hessian_apply(m, gpu(vv), ckpt=30, out_dtype=torch.float64))
    u, v = f32(vv[0]), f32(vv[1])
    assert np.all(np.isfinite(H))
    assert abs(np.vdot(u, H[1]) - np.vdot(H[0], v)) < 1e-3 * np.sqrt(np.vdot(u, H[0]) * np.vdot(v, H[1]))
    assert np.vdot(u, H[0]) > 0 and np.vdot(v, H[1]) > 0


def test_results_do_not_depend_on_workspace_contents(ragged):
    """Workspace memory arrives uninitialised: poisoning it with NaN bytes must not change anything."""
    w, P, _ = ragged
    m, v = gpu(w.m), gpu(w.v)
    dobs = gpu(synth.normal(5, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr))
    runs = {
        "hv": lambda: P.hessian_apply(m, v, ckpt=3),
        "hv_all": lambda: P.hessian_apply(m, v),
        "fwd": lambda: P.fwd_model(m),
        "born": lambda: P.born(m, v),
        "grad": lambda: P.misfit_grad(m, dobs, ckpt=2)[1],
    }
    for name, fn in runs.items():
        ref = host(fn())
        P._ws["ws"].fill_(255)                       # every float32 in the workspace becomes NaN
        again = host(fn())
        assert np.array_equal(ref, again), name
        assert np.all(np.isfinite(again)), name
