"""Posterior (Laplace approximation) objects and the gpCN step on the GPU
(hv_posterior_*, hv_gpcn_*) against the FP64 oracle (oracle/spd_oracle.py,
oracle/gpcn_oracle.py, oracle/lowrank_oracle.py, oracle/quadratic_oracle.py),
on the quadratic test model with the GPU's own operator and symbols."""
import numpy as np
import pytest
import torch

from oracle import gpcn_oracle as GO
from oracle import lowrank_oracle as LO
from oracle import quadratic_oracle as QO
from oracle import spd_oracle as SO
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300._lib import HV_QUAD_HD
from paper_2507_10804_gb300.hv import Posterior, Quad, approx_build_pdo_op, gpcn_accept, gpcn_propose
from tests._helpers import f32, rel

pytestmark = pytest.mark.gpu
NZ, NX, H = 40, 56, 10.0
LAM = [40.0, 30.0, 20.0, 12.0, 8.0, 5.0]
DELTA, GAMMA = 1.0, 2500.0
RHO0 = 0.12


@pytest.fixture(scope="module")
def model():
    Q = Quad(NZ, NX, H, LAM, DELTA, GAMMA, taper=4)
    D = approx_build_pdo_op(Q, RHO0, 8)
    S = D.sqrt()
    a, b = (x.cpu().numpy().astype(np.complex128) for x in S.symbol())
    return Q, D, S, a, b


def _normals(seed, k):
    v = synth.normal(seed, k * NZ * NX).reshape(k, NZ, NX)
    return f32(v).astype(np.float64), torch.tensor(v, dtype=torch.float32, device="cuda")


def _gpu_hd(Q):
    def f(X):
        Xt = torch.tensor(np.asarray(X), dtype=torch.float32, device="cuda")
        return Q.apply(Xt, HV_QUAD_HD).cpu().numpy().astype(np.float64)
    return f


def test_prior_only_posterior_is_closed_form():
    P = Posterior(NZ, NX, H, DELTA, GAMMA)
    n, nt = _normals(5, 2)
    z, it = P.sample(nt)
    assert it == 0
    z = z.cpu().numpy()
    Ro = P.apply(nt).cpu().numpy()
    x, it = P.solve(nt, rtol=1e-6)
    x = x.cpu().numpy()
    assert it <= 2                                         # R^-1 preconditions R exactly
    for j in range(2):
        assert rel(z[j], LO.prior_Ainv(n[j], H, DELTA, GAMMA)) < 2e-5
        assert rel(Ro[j], LO.prior_R(n[j], H, DELTA, GAMMA)) < 2e-5
        assert rel(x[j], LO.prior_Rinv(n[j], H, DELTA, GAMMA)) < 1e-4
    P.close()


def test_square_root_posterior_apply_solve_sample(model):
    Q, D, S, a, b = model
    P = Posterior(NZ, NX, H, DELTA, GAMMA, approx=S)
    H0 = lambda x: SO.spd_apply(a, b, x) + LO.prior_R(x, H, DELTA, GAMMA)
    v, vt = _normals(11, 2)
    got = P.apply(vt).cpu().numpy()
    for j in range(2):
        assert rel(got[j], H0(v[j])) < 2e-5, rel(got[j], H0(v[j]))
    x, it = P.solve(vt, rtol=1e-7)
    assert 0 < it < 1000
    x = x.cpu().numpy()
    for j in range(2):
        want = SO.solve(H0, v[j], precond=lambda y: LO.prior_Rinv(y, H, DELTA, GAMMA))
        assert rel(x[j], want) < 2e-4, rel(x[j], want)
    n1, n1t = _normals(12, 2)
    n2, n2t = _normals(13, 2)
    z, it = P.sample(n1t, n2t, rtol=1e-7)
    z = z.cpu().numpy()
    for j in range(2):
        want = SO.posterior_sample(a, b, n1[j], n2[j], H, DELTA, GAMMA)
        assert rel(z[j], want) < 2e-4, rel(z[j], want)
    P.close()


def test_solve_with_the_exact_operator_gives_the_map(model):
    Q, D, S, a, b = model
    q = QO.make(NZ, NX, H, LAM, L=4)
    mstar = synth.smoothed_normal_vectors(17, 1, NZ, NX, 3.0)[0]
    ms = torch.tensor(mstar, dtype=torch.float32, device="cuda")
    _, g0 = Q.objective(torch.zeros((1, NZ, NX), device="cuda"), ms)
    P = Posterior(NZ, NX, H, DELTA, GAMMA)
    x, it = P.solve(-g0, op=Q, rtol=1e-7)
    x = x.cpu().numpy()[0]
    rhs = -QO.objective(q, np.zeros((NZ, NX)), f32(mstar), DELTA, GAMMA)[1]
    want = SO.solve(lambda y: QO.apply_Hd(q, y) + LO.prior_R(y, H, DELTA, GAMMA), rhs,
                    precond=lambda y: LO.prior_Rinv(y, H, DELTA, GAMMA))
    assert rel(x, want) < 5e-4, rel(x, want)
    _, gx = QO.objective(q, x, f32(mstar), DELTA, GAMMA)
    assert np.linalg.norm(gx) < 1e-4 * np.linalg.norm(rhs)                    # the MAP point
    P.close()


def test_low_rank_correction_matches_oracle(model):
    Q, D, S, a, b = model
    P = Posterior(NZ, NX, H, DELTA, GAMMA, approx=S)
    k, rank = 14, 8
    omega, omegat = _normals(21, k)
    P.correct(Q, omegat, rank, rtol=1e-7)
    lam, V = P.eigs()
    hd = _gpu_hd(Q)
    H0 = lambda x: SO.spd_apply(a, b, x) + LO.prior_R(x, H, DELTA, GAMMA)
    solve = lambda y: SO.solve(H0, y, precond=lambda t: LO.prior_Rinv(t, H, DELTA, GAMMA))
    resid = lambda X: hd(X) - np.stack([SO.spd_apply(a, b, x) for x in X])
    Vo, lamo = SO.corrected_lowrank(resid, H0, solve, omega, rank)
    _, lam_all = SO.corrected_lowrank(resid, H0, solve, omega, k)
    gap = (lam_all[rank - 1] - lam_all[rank]) / abs(lam_all[0])
    np.testing.assert_allclose(lam, lamo, rtol=2e-3 * max(1.0, abs(lam_all[0] / lam_all[rank - 1])))
    tol = max(2e-3, 1e-5 / gap)
    v, vt = _normals(22, 2)
    got = P.apply(vt).cpu().numpy()
    n1, n1t = _normals(23, 2)
    n2, n2t = _normals(24, 2)
    z, _ = P.sample(n1t, n2t, rtol=1e-7)
    z = z.cpu().numpy()
    for j in range(2):
        want = SO.corrected_apply(H0, Vo, lamo, v[j])
        assert rel(got[j], want) < tol, (j, rel(got[j], want), tol)
        z0 = SO.posterior_sample(a, b, n1[j], n2[j], H, DELTA, GAMMA)
        want = SO.corrected_sample(H0, Vo, lamo, z0)
        assert rel(z[j], want) < tol, (j, rel(z[j], want), tol)
    P.close()


def test_gpcn_kernels_match_oracle():
    c = 4
    m, mt = _normals(31, c)
    mp, mpt = _normals(32, 1)
    zeta, zt = _normals(33, c)
    beta = 0.3
    m_new, d_new = gpcn_propose(mt, mpt[0].contiguous(), zt, beta)
    for j in range(c):
        want = GO.propose(m[j], mp[0], beta, zeta[j])
        assert rel(m_new[j].cpu().numpy(), want) < 1e-6
        assert rel(d_new[j].cpu().numpy(), want - mp[0]) < 1e-6
    Hd = torch.tensor(synth.normal(34, c * NZ * NX).reshape(c, NZ, NX), dtype=torch.float32, device="cuda")
    phi = torch.tensor([1.0, 2.0, -3.0, 0.5], dtype=torch.float64, device="cuda")
    dh = d_new.double().cpu().numpy()
    Hh = Hd.double().cpu().numpy()
    dnew = np.array([phi[j].item() - 0.5 * np.vdot(dh[j], Hh[j]) for j in range(c)])
    delta_cur = torch.tensor(dnew + np.array([5.0, -5.0, 0.0, 1.0]), dtype=torch.float64, device="cuda")
    log_u = torch.log(torch.tensor([0.5, 0.5, 0.5, 0.9], dtype=torch.float64, device="cuda"))
    before = mt.clone()
    dc = delta_cur.cpu().numpy().copy()
    acc = gpcn_accept(phi, m_new, d_new, Hd, log_u, mt, delta_cur).cpu().numpy()
    for j in range(c):
        want = GO.accept(dc[j], dnew[j], float(torch.exp(log_u[j])))
        assert bool(acc[j]) == want, j
        assert torch.equal(mt[j], m_new[j] if want else before[j])
        assert abs(delta_cur[j].item() - (dnew[j] if want else dc[j])) < 1e-9 * max(1.0, abs(dnew[j]))


def test_gpcn_chain_on_the_quadratic_model(model):
    """A short gpCN run with the corrected square-root PDO approximation: every step goes
    through the library (sample, propose, objective, H~ apply, accept)."""
    Q, D, S, a, b = model
    P = Posterior(NZ, NX, H, DELTA, GAMMA, approx=S)
    omega = torch.tensor(synth.normal(41, 12 * NZ * NX).reshape(12, NZ, NX), dtype=torch.float32, device="cuda")
    P.correct(Q, omega, 8)
    mstar = torch.tensor(synth.smoothed_normal_vectors(42, 1, NZ, NX, 3.0)[0], dtype=torch.float32, device="cuda")
    _, g0 = Q.objective(torch.zeros((1, NZ, NX), device="cuda"), mstar)
    m_map, _ = P.solve(-g0, op=Q, rtol=1e-7)
    c, steps, beta = 8, 30, 0.5
    gen = torch.Generator(device="cuda").manual_seed(7)
    m = m_map.repeat(c, 1, 1).contiguous()
    phi, _ = Q.objective(m, mstar, grad=False)
    delta = torch.empty(c, dtype=torch.float64, device="cuda")
    zero = torch.zeros_like(m)
    gpcn_accept(phi, m, zero, zero, torch.full((c,), -float("inf"), dtype=torch.float64, device="cuda"), m, delta)
    total = 0
    for _ in range(steps):
        n1 = torch.randn((c, NZ, NX), device="cuda", generator=gen)
        n2 = torch.randn((c, NZ, NX), device="cuda", generator=gen)
        zeta, _ = P.sample(n1, n2)
        m_new, d_new = gpcn_propose(m, m_map[0].contiguous(), zeta, beta)
        phi_new, _ = Q.objective(m_new, mstar, grad=False)
        Hd = P.apply(d_new)
        log_u = torch.log(torch.rand(c, dtype=torch.float64, device="cuda", generator=gen))
        total += int(gpcn_accept(phi_new, m_new, d_new, Hd, log_u, m, delta).sum())
    assert torch.isfinite(m).all() and torch.isfinite(delta).all()
    assert 0 < total <= c * steps
    P.close()


def test_posterior_calls_allocate_nothing_and_respect_max_k(model):
    """All scratch is sized at create for max_k fields: later calls allocate no device memory,
    and a call with more fields is rejected."""
    Q, D, S, a, b = model
    from paper_2507_10804_gb300._lib import HvError
    P = Posterior(NZ, NX, H, DELTA, GAMMA, approx=S, max_k=8)
    n1, n1t = _normals(31, 8)
    n2, n2t = _normals(32, 8)
    omega = torch.tensor(synth.normal(33, 8 * NZ * NX).reshape(8, NZ, NX), dtype=torch.float32, device="cuda")
    for rep in range(2):        # the first pass warms the operator's and torch's own caches
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        P.correct(Q, omega, 4, rtol=1e-6)
        z, _ = P.sample(n1t, n2t)
        x, _ = P.solve(n1t, rtol=1e-6)
        y = P.apply(n1t)
        torch.cuda.synchronize()
    # the outputs above are torch's (3 x 8 fields, reused from its cache); nothing else may appear
    assert torch.cuda.mem_get_info()[0] >= free0 - (2 << 20)
    assert torch.isfinite(z).all() and torch.isfinite(x).all() and torch.isfinite(y).all()
    big = torch.zeros((9, NZ, NX), dtype=torch.float32, device="cuda")
    with pytest.raises(HvError):
        P.solve(big)
    with pytest.raises(HvError):
        P.apply(big)
    P.close()
