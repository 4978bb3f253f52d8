"""Square-root (SPD) forms of the PDO and PSF+ approximations on the GPU
(hv_approx_sqrt_pdo, hv_approx_build_psfplus_sqrt, the SQRT / SQRT_T / H apply
modes) against the FP64 oracle (oracle/spd_oracle.py, oracle/psfplus_oracle.py)
fed the GPU's own PDO columns and PSFs."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import pdo_oracle as DO
from oracle import psfplus_oracle as PP
from oracle import spd_oracle as SO
from paper_2507_10804_gb300 import _lib, synth
from paper_2507_10804_gb300._lib import HV_APPROX_H, HV_APPROX_INVSQRT, HV_APPROX_SQRT, HV_APPROX_SQRT_T
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem, psf_plus
from tests._helpers import f32, ragged_workload, rel

pytestmark = pytest.mark.gpu
RHO0 = 0.15


@pytest.fixture(scope="module")
def built():
    w = ragged_workload(nz=37, nx=71, nb=6, nt=150, ns=3, nr=7)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    A = P.approx_build_psf(m, 8, 4, ckpt=HV_CKPT_ALL)
    D = P.approx_build_pdo(m, RHO0, 8, ckpt=HV_CKPT_ALL)
    return w, P, m, A, D


def _vecs(w, seed, k=3):
    v = synth.smoothed_normal_vectors(seed, k, w.nz, w.nx, 1.5)
    return v, torch.tensor(v, dtype=torch.float32, device="cuda")


def test_pdo_square_root_matches_oracle(built):
    w, P, m, A, D = built
    Q = D.sqrt()
    assert Q.info["kind"] == 1 and Q.info["spd"] == 1 and D.info["spd"] == 0
    cols = D.symbol()[0].cpu().numpy().astype(np.complex128)
    a, b = SO.pdo_sqrt(cols, w.h, RHO0, 8)
    ga, gb = (x.cpu().numpy().astype(np.complex128) for x in Q.symbol())
    assert np.abs(ga - a).max() < 1e-6 * np.abs(a).max()
    assert np.abs(gb - b).max() < 1e-5 * np.abs(b).max()
    v, vt = _vecs(w, 61)
    vd = f32(v).astype(np.float64)
    for mode, want in ((HV_APPROX_SQRT, DO.lr_apply(a, b, vd)), (HV_APPROX_SQRT_T, SO.lr_apply_T(a, b, vd)),
                       (HV_APPROX_H, SO.spd_apply(a, b, vd))):
        got = Q.apply(vt, mode).cpu().numpy()
        for j in range(3):
            assert rel(got[j], want[j]) < 1e-5, (mode, j, rel(got[j], want[j]))
    Q.close()


def test_transpose_and_gram_properties(built):
    w, P, m, A, D = built
    Q = D.sqrt()
    v, vt = _vecs(w, 62, 2)
    Bv = Q.apply(vt[:1], HV_APPROX_SQRT).double()
    BTw = Q.apply(vt[1:], HV_APPROX_SQRT_T).double()
    lhs, rhs = float((vt[1:].double() * Bv).sum()), float((BTw * vt[:1].double()).sum())
    assert abs(lhs - rhs) < 1e-5 * (abs(lhs) + abs(rhs))
    G = Q.apply(vt).double()
    assert float((G * vt.double()).sum(dim=(1, 2)).min()) > 0                   # B B^T is PSD
    Q.close()


@pytest.mark.parametrize("tol", [1e-2, 1e-3])
def test_psfplus_square_root_matches_oracle(built, tol):
    w, P, m, A, D = built
    C = psf_plus(A, D, tol, spd=True)
    assert C.info["kind"] == 2 and C.info["spd"] == 1
    psf = A.psfs().cpu().numpy().astype(np.float64)
    cols = D.symbol()[0].cpu().numpy().astype(np.complex128)
    a, b, _, _ = PP.psf_plus(psf, 8, 2, cols, w.h, RHO0, 8, tol=tol, spd=True)
    assert C.info["r"] == a.shape[0]
    v, vt = _vecs(w, 63, 2)
    vd = f32(v).astype(np.float64)
    got = C.apply(vt).cpu().numpy()
    want = SO.spd_apply(a, b, vd)
    for j in range(2):
        assert rel(got[j], want[j]) < 1e-4, (tol, j, rel(got[j], want[j]))
    C.close()


def test_modes_are_validated(built):
    w, P, m, A, D = built
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    v = torch.zeros((1, w.nz, w.nx), dtype=torch.float32, device="cuda")
    o = torch.empty_like(v)
    for obj, mode in ((A, HV_APPROX_SQRT), (D, HV_APPROX_SQRT), (D, HV_APPROX_SQRT_T)):
        assert lib.hv_approx_apply(obj._a, v.data_ptr(), 1, o.data_ptr(), mode, stream) == _lib.HV_ENOTSUP
    Q = D.sqrt()
    assert lib.hv_approx_apply(Q._a, v.data_ptr(), 1, o.data_ptr(), HV_APPROX_INVSQRT, stream) == _lib.HV_ENOTSUP
    assert lib.hv_approx_apply(Q._a, v.data_ptr(), 1, o.data_ptr(), 4, stream) == _lib.HV_EINVAL
    out = ctypes.c_void_p(1)
    assert lib.hv_approx_sqrt_pdo(Q._a, ctypes.byref(out), stream) == _lib.HV_EINVAL      # already a square root
    assert out.value is None
    assert lib.hv_approx_sqrt_pdo(A._a, ctypes.byref(out), stream) == _lib.HV_EINVAL      # not a PDO object
    Q.close()
