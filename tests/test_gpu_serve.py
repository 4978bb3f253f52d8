"""Serving: requests from many clients on grids of different sizes are
admitted by memory budget and run concurrently; each result is bitwise the
same alone and in the mix."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import Problem
from paper_2507_10804_gb300._lib import HV_REQ_QUEUED
from paper_2507_10804_gb300.serve import Server
from tests._helpers import f32, oracle_problem, rel

pytestmark = pytest.mark.gpu


def make(nz, nx, ns, nt, seed):
    w = synth.workload(1, nt=nt)
    m = synth.gradient_grf_model(seed, nz, nx, 10.0)
    acq = synth.surface_acquisition(nx, ns, nx // 2)
    w = synth.Workload(name=f"{nz}x{nx}", nz=nz, nx=nx, nb=20, h=10.0, nt=nt, dt=synth.cfl_dt(10.0, float(m.max())),
                       f0=15.0, t0=0.1, vmax=float(m.max()), acq=acq, m=m,
                       v=synth.smoothed_normal_vectors(seed + 1, 2, nz, nx))
    return w, Problem.from_workload(w)


def t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def problems():
    return [make(48, 64, 4, 300, 11), make(96, 80, 6, 400, 12)]


def requests(problems, n=24, seed=7):
    u = synth.uniform(seed, 3 * n)
    out = []
    for i in range(n):
        w, P = problems[int(u[3 * i] * len(problems))]
        kind = ("hv", "grad", "misfit")[min(int(u[3 * i + 1] * 5) // 2, 2)]   # 40% / 40% / 20%
        m = w.m * (1.0 + 0.01 * synth.smoothed_normal_vectors(seed + 100 + i, 1, w.nz, w.nx, 4.0)[0])
        dobs = synth.normal(seed + 200 + i, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr) * 1e-3
        out.append((kind, w, P, t(m), t(w.v[:1 + i % 2]), t(dobs), 1 + (i % 3) * 5))
    return out


def run_direct(kind, w, P, m, v, dobs, ckpt):
    if kind == "hv":
        return [P.hessian_apply(m, v, ckpt=ckpt)]
    if kind == "grad":
        phi, g = P.misfit_grad(m, dobs, ckpt=ckpt)
        return [phi, g]
    phi, g = P.misfit_grad(m, dobs, ckpt=ckpt)
    return [phi]


def submit(S, kind, w, P, m, v, dobs, ckpt):
    if kind == "hv":
        rid, out = S.submit_hv(P, m, v, ckpt=ckpt)
        return rid, [out]
    if kind == "grad":
        rid, phi, g = S.submit_grad(P, m, dobs, ckpt=ckpt)
        return rid, [phi, g]
    rid, phi = S.submit_misfit(P, m, dobs)
    return rid, [phi]


def test_mixed_requests_equal_direct_calls_bitwise(problems):
    reqs = requests(problems)
    direct = [[x.cpu().numpy() for x in run_direct(*r)] for r in reqs]
    S = Server(hbm_budget=2 << 30, max_concurrent=8)
    subs = [submit(S, *r) for r in reqs]                       # all arrive while others run
    for (rid, outs), ref in zip(subs, direct):
        assert S.wait(rid, timeout=300) == 0
        for o, r_ in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r_)
    infos = [S.info(rid) for rid, _ in subs]
    starts = sorted(i["t_start"] for i in infos)
    dones = sorted(i["t_done"] for i in infos)
    assert starts[1] < dones[0]                                 # requests overlapped on the device
    S.close()


def test_tight_budget_queues_and_rejects(problems):
    reqs = requests(problems, n=8, seed=9)
    op = {"hv": 4, "grad": 3, "misfit": 6}
    need = max(P.workspace_size(op[kind], v.shape[0] if kind == "hv" else 1, ckpt)
               for kind, w, P, m, v, dobs, ckpt in reqs)
    S = Server(hbm_budget=need + 4096, max_concurrent=4)        # room for about one request
    subs = [submit(S, *r) for r in reqs]
    for rid, _ in subs:
        assert S.wait(rid, timeout=300) == 0
    with pytest.raises(Exception):
        big = make(160, 160, 8, 500, 13)[1]
        S.submit_hv(big, t(np.full((160, 160), 2000.0)), t(np.zeros((64, 160, 160))), ckpt=-1)
    S.close()


def test_misfit_matches_oracle(problems):
    w, P = problems[0]
    dobs = synth.normal(5, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr) * 1e-3
    S = Server(hbm_budget=1 << 30, max_concurrent=2)
    rid, phi = S.submit_misfit(P, t(w.m), t(dobs))
    assert S.wait(rid) == 0
    ref = O.misfit_grad(oracle_problem(w), f32(w.m), f32(dobs))[0]
    assert abs(float(phi) - ref) < 2e-4 * ref
    S.close()


def test_approximate_hessian_requests_in_the_mix(problems):
    """Apply requests of built PSF and PDO approximations run among H v requests
    (applies of one PDO object on different streams run one after another); every
    result is bitwise that of the direct call."""
    (w0, P0), (w1, P1) = problems
    A = P0.approx_build_psf(t(w0.m), 8, 4, ckpt=5)
    D = P0.approx_build_pdo(t(w0.m), 0.15, 8, ckpt=5)
    vs = [t(synth.smoothed_normal_vectors(300 + i, 1 + i % 3, w0.nz, w0.nx, 1.5)) for i in range(6)]
    objs = [A if i % 2 == 0 else D for i in range(6)]
    direct_a = [o.apply(v).cpu().numpy() for o, v in zip(objs, vs)]
    direct_h = P1.hessian_apply(t(w1.m), t(w1.v[:1]), ckpt=6).cpu().numpy()
    S = Server(hbm_budget=1 << 30, max_concurrent=4)
    rh, oh = S.submit_hv(P1, t(w1.m), t(w1.v[:1]), ckpt=6)
    subs = [S.submit_approx(o, v) for o, v in zip(objs, vs)]
    assert S.wait(rh, timeout=300) == 0
    assert np.array_equal(oh.cpu().numpy(), direct_h)
    for (rid, out), ref in zip(subs, direct_a):
        assert S.wait(rid, timeout=300) == 0
        assert np.array_equal(out.cpu().numpy(), ref)
        assert S.info(rid)["kind"] == 3
    S.close()
    A.close()
    D.close()


def test_approximation_modes_in_the_mix(problems):
    """LR sampling-factor and H~_d requests and square-root PDO requests on several streams at
    once: the shared scratch of each object is ordered across streams, so every result is bitwise
    that of the direct call; an unknown mode is rejected at submission."""
    from paper_2507_10804_gb300._lib import HV_APPROX_H, HV_APPROX_INVSQRT, HV_APPROX_SQRT, HV_APPROX_SQRT_T
    w0, P0 = problems[0]
    omega = t(synth.normal(401, 8 * w0.nz * w0.nx).reshape(8, w0.nz, w0.nx))
    L = P0.approx_build_lr(t(w0.m), 1.0, 2500.0, 6, omega, ckpt=5)
    Q = P0.approx_build_pdo(t(w0.m), 0.15, 8, ckpt=5).sqrt()
    jobs = []
    for i in range(12):
        v = t(synth.smoothed_normal_vectors(410 + i, 1 + i % 2, w0.nz, w0.nx, 1.5))
        obj, mode = [(L, HV_APPROX_INVSQRT), (L, HV_APPROX_H), (Q, HV_APPROX_SQRT), (Q, HV_APPROX_SQRT_T)][i % 4]
        jobs.append((obj, mode, v, obj.apply(v, mode).cpu().numpy()))
    S = Server(hbm_budget=1 << 30, max_concurrent=4)
    subs = [S.submit_approx(o, v, mode) for o, mode, v, _ in jobs]
    for (rid, out), (_, _, _, ref) in zip(subs, jobs):
        assert S.wait(rid, timeout=300) == 0
        assert np.array_equal(out.cpu().numpy(), ref)
    with pytest.raises(Exception):
        S.submit_approx(L, jobs[0][2], 7)
    S.close()
    L.close()
    Q.close()


def test_merged_call_equals_separate_calls_bitwise(problems):
    """hv_apply_batch: H v entries, gradients and misfits at one model share one forward sweep;
    every output is bitwise that of its separate call (and a misfit-only batch too)."""
    w, P = problems[0]
    m = t(w.m)
    v1, v2 = t(w.v[:1]), t(w.v[:2])
    d1 = t(synth.normal(61, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr) * 1e-3)
    d2 = t(synth.normal(62, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr) * 1e-3)
    ref_h = [P.hessian_apply(m, v, ckpt=5).cpu().numpy() for v in (v1, v2)]
    ref_g = [[x.cpu().numpy() for x in P.misfit_grad(m, d, ckpt=5)] for d in (d1, d2)]
    ref_m = P.misfit(m, d2).cpu().numpy()
    hv, gr, mi = P.apply_batch(m, hv=[v1, v2], grads=[d1, d2], misfits=[d2], ckpt=5)
    for a, b in zip(hv, ref_h):
        assert np.array_equal(a.cpu().numpy(), b)
    for (phi, g), (rphi, rg) in zip(gr, ref_g):
        assert np.array_equal(phi.cpu().numpy(), rphi) and np.array_equal(g.cpu().numpy(), rg)
    assert np.array_equal(mi[0].cpu().numpy(), ref_m)
    _, _, only = P.apply_batch(m, misfits=[d1, d2])
    assert np.array_equal(only[1].cpu().numpy(), ref_m)


def test_queued_requests_on_one_model_run_as_one_call(problems):
    """Continuous batching: requests queued behind a running one, on one problem and model, are
    admitted together as one merged call (info()["batch"]) with results bitwise equal to direct calls;
    with batching off the same requests run one by one."""
    (w, P), (w2, P2) = problems
    m = t(w.m)
    vs = [t(w.v[:1]), t(w.v[1:2])]
    d = t(synth.normal(71, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr) * 1e-3)
    ref_h = [P.hessian_apply(m, v, ckpt=5).cpu().numpy() for v in vs]
    ref_phi, ref_g = (x.cpu().numpy() for x in P.misfit_grad(m, d, ckpt=5))
    ref_m = P.misfit(m, d).cpu().numpy()
    for batching in (64, 0):
        S = Server(hbm_budget=2 << 30, max_concurrent=1)
        S.set_engine(0)                                   # the misfit runs as a call, not in a lane
        S.set_batching(batching)
        blocker, _ = S.submit_hv(P2, t(w2.m), t(w2.v), ckpt=1)        # about 80k recomputed steps
        (r1, o1), (r2, o2) = (S.submit_hv(P, m, v, ckpt=5) for v in vs)
        r3, phi, g = S.submit_grad(P, m, d, ckpt=5)
        r4, phm = S.submit_misfit(P, m, d)
        for rid in (blocker, r1, r2, r3, r4):
            assert S.wait(rid, timeout=300) == 0
        assert S.info(blocker)["batch"] == 1
        assert [S.info(r)["batch"] for r in (r1, r2, r3, r4)] == ([4] * 4 if batching else [1] * 4)
        assert np.array_equal(o1.cpu().numpy(), ref_h[0]) and np.array_equal(o2.cpu().numpy(), ref_h[1])
        assert np.array_equal(phi.cpu().numpy(), ref_phi) and np.array_equal(g.cpu().numpy(), ref_g)
        assert np.array_equal(phm.cpu().numpy(), ref_m)
        S.close()


def test_interleaved_queue_merges_every_request_once(problems):
    """Requests on two problems queued alternately behind a running one: each admission merges the
    queued requests of one problem out of the middle of the queue; every request completes exactly once
    with its direct result."""
    (w, P), (w2, P2) = problems
    m, m2 = t(w.m), t(w2.m)
    vs = [t(w.v[i % 2:i % 2 + 1]) for i in range(6)]
    vs2 = [t(w2.v[i % 2:i % 2 + 1]) for i in range(6)]
    ref = [P.hessian_apply(m, v, ckpt=5).cpu().numpy() for v in vs]
    ref2 = [P2.hessian_apply(m2, v, ckpt=4).cpu().numpy() for v in vs2]
    S = Server(hbm_budget=4 << 30, max_concurrent=2)
    blockers = [S.submit_hv(P2, m2, t(w2.v), ckpt=1)[0] for _ in range(2)]     # both streams busy
    subs = []
    for i in range(6):
        subs.append((S.submit_hv(P, m, vs[i], ckpt=5), ref[i]))
        subs.append((S.submit_hv(P2, m2, vs2[i], ckpt=4), ref2[i]))
    for rid in blockers:
        assert S.wait(rid, timeout=300) == 0
    for (rid, out), r in subs:
        assert S.wait(rid, timeout=300) == 0
        assert np.array_equal(out.cpu().numpy(), r)
    assert sum(S.info(rid)["batch"] > 1 for (rid, _), _ in subs) >= 6
    S.close()


def test_queued_approximation_applies_merge_bitwise(problems):
    """Applies of one approximation in one mode queued behind a running request run as one apply of all
    their vectors; each result is bitwise that of its own direct apply (PSF, PDO through cuFFT, the square-root
    PDO's three modes, and the low-rank approximation's H~ and sampling factor, whose prior inverse runs cuFFT)."""
    from paper_2507_10804_gb300._lib import HV_APPROX_H, HV_APPROX_INVSQRT, HV_APPROX_SQRT, HV_APPROX_SQRT_T
    (w0, P0), (w1, P1) = problems
    m0 = t(w0.m)
    A = P0.approx_build_psf(m0, 8, 4, ckpt=5)
    D = P0.approx_build_pdo(m0, 0.15, 8, ckpt=5)
    Q = D.sqrt()
    omega = t(synth.normal(501, 8 * w0.nz * w0.nx).reshape(8, w0.nz, w0.nx))
    L = P0.approx_build_lr(m0, 1.0, 2500.0, 6, omega, ckpt=5)
    cases = [(A, HV_APPROX_H), (D, HV_APPROX_H), (Q, HV_APPROX_H), (Q, HV_APPROX_SQRT), (Q, HV_APPROX_SQRT_T),
             (L, HV_APPROX_H), (L, HV_APPROX_INVSQRT)]
    S = Server(hbm_budget=2 << 30, max_concurrent=1)
    for obj, mode in cases:
        vs = [t(synth.smoothed_normal_vectors(600 + i, 1 + i % 2, w0.nz, w0.nx, 1.5)) for i in range(5)]
        direct = [obj.apply(v, mode).cpu().numpy() for v in vs]
        blocker, _ = S.submit_hv(P1, t(w1.m), t(w1.v), ckpt=1)
        subs = [S.submit_approx(obj, v, mode) for v in vs]
        assert S.wait(blocker, timeout=300) == 0
        for (rid, out), ref in zip(subs, direct):
            assert S.wait(rid, timeout=300) == 0
            assert np.array_equal(out.cpu().numpy(), ref), (obj.info["kind"], mode)
        assert all(S.info(rid)["batch"] == 5 for rid, _ in subs), [S.info(rid)["batch"] for rid, _ in subs]
    S.close()
    for o in (A, D, Q, L):
        o.close()


def test_queued_misfits_at_different_models_run_as_one_sweep(problems):
    """Misfit requests on one problem at different models (MCMC chains' proposals) queued behind a running
    request run as one sweep of all their models (hv_misfit_models); each phi is bitwise the direct misfit."""
    (w0, P0), (w1, P1) = problems
    dobs = t(synth.normal(211, w0.ns * w0.nt * w0.nr).reshape(w0.ns, w0.nt, w0.nr) * 1e-3)
    z = synth.smoothed_normal_vectors(213, 6, w0.nz, w0.nx, 4.0)
    ms = [t(np.minimum(w0.m * (1.0 + 0.03 * z[i] / np.abs(z[i]).max()), w0.vmax)) for i in range(6)]
    direct = [float(P0.misfit(m, dobs)) for m in ms]
    S = Server(hbm_budget=2 << 30, max_concurrent=1)
    S.set_engine(0)                                       # misfits run as calls, not in a lane
    blocker, _ = S.submit_hv(P1, t(w1.m), t(w1.v), ckpt=1)
    subs = [S.submit_misfit(P0, m, dobs) for m in ms]
    assert S.wait(blocker, timeout=300) == 0
    for (rid, phi), ref in zip(subs, direct):
        assert S.wait(rid, timeout=300) == 0
        assert float(phi) == ref
    assert [S.info(rid)["batch"] for rid, _ in subs] == [6] * 6
    S.close()


@pytest.mark.parametrize("device_loop", [False, True])
def test_misfits_join_a_running_lane_at_the_next_time_step(device_loop):
    """Misfit lanes, ticked by the server's thread or served by the engine's device-resident loop: misfits
    submitted while another misfit on the same problem is running join the problem's lane at its next time
    step instead of waiting for that sweep to end (their runs overlap); each phi is bitwise the direct misfit,
    and the lane's occupancy at each join is reported."""
    import time
    w, P = make(48, 64, 4, 3000, 17)                      # a 3000-step sweep: tens of milliseconds
    dobs = t(synth.normal(221, w.ns * w.nt * w.nr).reshape(w.ns, w.nt, w.nr) * 1e-3)
    z = synth.smoothed_normal_vectors(223, 3, w.nz, w.nx, 4.0)
    ms = [t(np.minimum(w.m * (1.0 + 0.03 * z[i] / np.abs(z[i]).max()), w.vmax)) for i in range(3)]
    direct = [float(P.misfit(m, dobs)) for m in ms]
    S = Server(hbm_budget=2 << 30, max_concurrent=2)
    S.set_engine_loop(device_loop)
    a, pa = S.submit_misfit(P, ms[0], dobs)
    t0 = time.perf_counter()
    while S.poll(a) == HV_REQ_QUEUED and time.perf_counter() - t0 < 60:
        time.sleep(1e-4)
    b, pb = S.submit_misfit(P, ms[1], dobs)
    c, pc = S.submit_misfit(P, ms[2], dobs)
    for rid in (a, b, c):
        assert S.wait(rid, timeout=300) == 0
    ia, ib, ic = S.info(a), S.info(b), S.info(c)
    assert ib["t_start"] < ia["t_done"] and ic["t_start"] < ia["t_done"], (ia, ib, ic)   # joined mid-sweep
    assert (ia["batch"], ib["batch"], ic["batch"]) == (1, 2, 3)
    assert [float(pa), float(pb), float(pc)] == direct
    S.close()
