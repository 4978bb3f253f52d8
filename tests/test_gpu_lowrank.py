"""Matern prior operator and the low-rank approximation on the GPU against the
FP64 oracle (oracle/lowrank_oracle.py): A, A^-1, R, R^-1; the randomized double
pass with the same test matrix and the same Hessian (the GPU's, passed to the
oracle as a function), its eigenvalues, the approximate Hessian and the
posterior sampling factor."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import lowrank_oracle as LO
from paper_2507_10804_gb300 import _lib, synth
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem, prior_apply
from tests._helpers import f32, ragged_workload, rel

pytestmark = pytest.mark.gpu
DELTA, GAMMA = 1.0, 2500.0          # correlation length ~ sqrt(gamma / delta) = 50 m on the 10 m grid


@pytest.mark.parametrize("nz,nx", [(37, 71), (64, 64), (5, 9)])
def test_prior_operators_match_oracle(nz, nx):
    v = synth.smoothed_normal_vectors(3, 2, nz, nx, 1.0)
    vt = torch.tensor(v, dtype=torch.float32, device="cuda")
    ops = [LO.prior_A, LO.prior_Ainv, LO.prior_R, LO.prior_Rinv]
    for op, f in enumerate(ops):
        got = prior_apply(vt, 10.0, DELTA, GAMMA, op).cpu().numpy()
        for j in range(2):
            want = f(f32(v[j]), 10.0, DELTA, GAMMA)
            assert rel(got[j], want) < 2e-5, (op, j, rel(got[j], want))


@pytest.fixture(scope="module")
def problem():
    w = ragged_workload(nz=37, nx=71, nb=6, nt=150, ns=3, nr=7)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    return w, P, m


@pytest.mark.parametrize("rank", [10, 6])
def test_lowrank_matches_oracle_on_the_same_hessian(problem, rank):
    """rank = k: no truncation, the two sides agree to FP32 rounding.  rank < k: the kept
    eigenvectors move with the rounding by about eps lambda_1 / (lambda_r - lambda_r+1)
    (Davis-Kahan), so the bound is taken from the oracle's own spectrum."""
    w, P, m = problem
    k = 10
    omega = synth.normal(77, k * w.nz * w.nx).reshape(k, w.nz, w.nx)
    A = P.approx_build_lr(m, DELTA, GAMMA, rank, torch.tensor(omega, dtype=torch.float32, device="cuda"),
                          ckpt=HV_CKPT_ALL)
    assert A.info["kind"] == 3 and A.info["r"] == rank
    lam, V = A.eigs()

    def gpu_hessian(X):
        Xt = torch.tensor(np.asarray(X), dtype=torch.float32, device="cuda")
        return P.hessian_apply(m, Xt, ckpt=HV_CKPT_ALL).cpu().numpy().astype(np.float64)

    Vo, lamo = LO.lowrank(gpu_hessian, f32(omega), rank, w.h, DELTA, GAMMA)
    _, lam_all = LO.lowrank(gpu_hessian, f32(omega), k, w.h, DELTA, GAMMA)
    gap = (lam_all[rank - 1] - lam_all[rank]) / lam_all[0] if rank < k else 1.0
    tol = max(1e-4, 1e-6 / gap)
    np.testing.assert_allclose(lam, lamo, rtol=1e-4 * max(1.0, lam_all[0] / lam_all[rank - 1]))
    x = synth.smoothed_normal_vectors(78, 2, w.nz, w.nx, 1.5)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    got_h, got_s = A.apply(xt).cpu().numpy(), A.sample_factor(xt).cpu().numpy()
    for j in range(2):
        want_h = LO.apply_H(Vo, lamo, f32(x[j]), w.h, DELTA, GAMMA)
        want_s = LO.apply_sample_factor(Vo, lamo, f32(x[j]), w.h, DELTA, GAMMA)
        assert rel(got_h[j], want_h) < tol, (rank, j, rel(got_h[j], want_h), tol)
        assert rel(got_s[j], want_s) < tol, (rank, j, rel(got_s[j], want_s), tol)
    # V^T R V = I on the GPU factors
    Vn = V.cpu().numpy().astype(np.float64)
    RV = np.stack([LO.prior_R(v, w.h, DELTA, GAMMA) for v in Vn])
    np.testing.assert_allclose(Vn.reshape(rank, -1) @ RV.reshape(rank, -1).T, np.eye(rank), atol=1e-3)
    A.close()


def test_lowrank_arguments_are_validated(problem):
    w, P, m = problem
    lib = _lib.load()
    out = ctypes.c_void_p(1)
    omega = torch.randn((4, w.nz, w.nx), device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hv_approx_build_lr(P._h, m.data_ptr(), ctypes.c_double(DELTA), ctypes.c_double(GAMMA), 5,
                                  omega.data_ptr(), 4, 5, ctypes.byref(out), ws.data_ptr(), ws.numel(),
                                  stream) == _lib.HV_EINVAL                       # rank > k
    assert out.value is None
    assert lib.hv_approx_build_lr(P._h, m.data_ptr(), ctypes.c_double(DELTA), ctypes.c_double(GAMMA), 2,
                                  omega.data_ptr(), 4, 5, ctypes.byref(out), ws.data_ptr(), 1024,
                                  stream) == _lib.HV_ENOMEM
    A = P.approx_build_lr(m, DELTA, GAMMA, 2, omega, ckpt=5)
    v = torch.zeros((1, w.nz, w.nx), dtype=torch.float32, device="cuda")
    o = torch.empty_like(v)
    assert lib.hv_approx_apply(A._a, v.data_ptr(), 1, o.data_ptr(), 1, stream) == _lib.HV_ENOTSUP
    assert lib.hv_prior_apply(8, 8, ctypes.c_double(10.0), ctypes.c_double(0.0), ctypes.c_double(1.0), v.data_ptr(),
                              1, o.data_ptr(), 0, stream) == _lib.HV_EINVAL      # delta must be > 0
    A.close()
