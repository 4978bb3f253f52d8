"""The quadratic test model on the GPU (hv_quad_*) against the FP64 oracle
(oracle/quadratic_oracle.py), and approximations built through the operator
interface (hv_approx_build_*_op) from it, against the oracle builds fed the
GPU's own operator."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import lowrank_oracle as LO
from oracle import pdo_oracle as DO
from oracle import psf_oracle as PO
from oracle import quadratic_oracle as QO
from paper_2507_10804_gb300 import _lib, synth
from paper_2507_10804_gb300._lib import HV_QUAD_A, HV_QUAD_AT, HV_QUAD_HD, HV_QUAD_HD_RAW
from paper_2507_10804_gb300.hv import Quad, approx_build_lr_op, approx_build_pdo_op, approx_build_psf_op
from tests._helpers import f32, rel

pytestmark = pytest.mark.gpu
NZ, NX, H = 48, 70, 10.0
LAM = [40.0, 30.0, 20.0, 12.0, 8.0, 5.0]
DELTA, GAMMA = 1.0, 2500.0


@pytest.fixture(scope="module")
def quad():
    Q = Quad(NZ, NX, H, LAM, DELTA, GAMMA, taper=5)
    q = QO.make(NZ, NX, H, LAM, L=5)
    return Q, q


def _vecs(seed, k):
    v = synth.smoothed_normal_vectors(seed, k, NZ, NX, 1.5)
    return f32(v).astype(np.float64), torch.tensor(v, dtype=torch.float32, device="cuda")


def test_tables_match_oracle(quad):
    Q, q = quad
    a, b, V, W = (x.cpu().numpy() for x in Q.tables())
    assert np.abs(a.imag).max() == 0 and np.abs(b.imag).max() == 0
    assert np.abs(a.real - q.a).max() < 1e-6 * np.abs(q.a).max()
    assert np.abs(b.real - q.b).max() < 1e-6 * np.abs(q.b).max()
    assert np.abs(V - q.V).max() < 1e-6 * np.abs(q.V).max()
    assert np.abs(W - q.W).max() < 1e-6


@pytest.mark.parametrize("op,fn", [(HV_QUAD_A, QO.apply_A), (HV_QUAD_AT, QO.apply_AT),
                                   (HV_QUAD_HD_RAW, QO.apply_Hd_raw), (HV_QUAD_HD, QO.apply_Hd)])
def test_applies_match_oracle(quad, op, fn):
    Q, q = quad
    v, vt = _vecs(71 + op, 3)
    got = Q.apply(vt, op).cpu().numpy()
    want = fn(q, v)
    for j in range(3):
        assert rel(got[j], want[j]) < 2e-5, (op, j, rel(got[j], want[j]))


@pytest.mark.parametrize("one_target", [True, False])
def test_objective_matches_oracle(quad, one_target):
    Q, q = quad
    m, mt = _vecs(81, 3)
    s, st = _vecs(82, 1 if one_target else 3)
    phi, g = Q.objective(mt, st[0] if one_target else st)
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    for j in range(3):
        want_phi, want_g = QO.objective(q, m[j], s[0] if one_target else s[j], DELTA, GAMMA)
        assert abs(phi[j] - want_phi) < 1e-5 * abs(want_phi), (j, phi[j], want_phi)
        assert rel(g[j], want_g) < 2e-5, (j, rel(g[j], want_g))


def _gpu_hd(Q):
    def f(X):
        Xt = torch.tensor(np.asarray(X), dtype=torch.float32, device="cuda")
        return Q.apply(Xt, HV_QUAD_HD).cpu().numpy().astype(np.float64)
    return f


def test_operator_builds_match_oracle_on_the_same_operator(quad):
    Q, q = quad
    hd = _gpu_hd(Q)
    # PSF: the PSFs are the windows of the operator applied to the impulse batches
    A = approx_build_psf_op(Q, 8, 4)
    assert A.info["kind"] == 0
    want = PO.build(hd, NZ, NX, 8, 2)
    got = A.psfs().cpu().numpy()
    assert np.abs(got - want).max() < 1e-5 * np.abs(want).max()
    A.close()
    # PDO: columns from the operator applied to the probe
    rho0 = 0.12
    D = approx_build_pdo_op(Q, rho0, 8)
    a = D.symbol()[0].cpu().numpy().astype(np.complex128)
    Hvp = hd(DO.probe(NZ, NX, H, rho0, 8)[None])[0]
    want_a = DO.extract_columns(Hvp, H, rho0, 8)
    for k in range(8):
        assert rel(a[k], want_a[k]) < 1e-5, (k, rel(a[k], want_a[k]))
    D.close()
    # LR: eigenvalues of the double pass on the same operator
    omega = synth.normal(91, 12 * NZ * NX).reshape(12, NZ, NX)
    L = approx_build_lr_op(Q, DELTA, GAMMA, 12, torch.tensor(omega, dtype=torch.float32, device="cuda"))
    lam, _ = L.eigs()
    _, lamo = LO.lowrank(hd, f32(omega), 12, H, DELTA, GAMMA)
    np.testing.assert_allclose(lam, lamo, rtol=1e-4)
    L.close()


def test_quad_arguments_are_validated():
    lib = _lib.load()
    q = ctypes.c_void_p(1)
    lam = (ctypes.c_double * 2)(1.0, 2.0)
    assert lib.hv_quad_create(NZ, NX, H, 0.1, 5, 3, lam, DELTA, GAMMA, ctypes.byref(q)) == _lib.HV_EINVAL   # odd
    assert q.value is None
    assert lib.hv_quad_create(NZ, NX, H, -1.0, 5, 2, lam, DELTA, GAMMA, ctypes.byref(q)) == _lib.HV_EINVAL
    assert lib.hv_quad_create(NZ, NX, H, 0.1, 30, 2, lam, DELTA, GAMMA, ctypes.byref(q)) == _lib.HV_EINVAL
    bad = (ctypes.c_double * 2)(1.0, -2.0)
    assert lib.hv_quad_create(NZ, NX, H, 0.1, 5, 2, bad, DELTA, GAMMA, ctypes.byref(q)) == _lib.HV_EINVAL
    Q = Quad(NZ, NX, H, [], DELTA, GAMMA)                         # no low-rank part is allowed
    v = torch.zeros((1, NZ, NX), device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hv_quad_apply(Q._q, 7, v.data_ptr(), 1, v.data_ptr(), stream) == _lib.HV_EINVAL
    assert float(Q.apply(v).abs().max()) == 0.0
    op = _lib.HvOperator()
    assert lib.hv_approx_build_pdo_op(ctypes.byref(op), ctypes.c_double(0.1), 8, ctypes.byref(q), stream) == _lib.HV_EINVAL
    Q.close()
