"""PSF+ on the GPU (hv_approx_build_psfplus) against the FP64 oracle
(oracle/psfplus_oracle.py) fed the GPU's own PSFs and PDO columns: the rank,
the symbol A B (compared through applies: the SVD basis is fixed only up to
phases) and the argument checks."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import pdo_oracle as DO
from oracle import psfplus_oracle as PP
from paper_2507_10804_gb300 import _lib, synth
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


@pytest.mark.parametrize("tol", [1e-1, 1e-2, 1e-3])
def test_psfplus_matches_oracle_on_the_same_inputs(built, tol):
    w, P, m, A, D = built
    C = psf_plus(A, D, tol)
    psf = A.psfs().cpu().numpy().astype(np.float64)
    cols = D.symbol()[0].cpu().numpy().astype(np.complex128)
    a, b, alpha, a0 = PP.psf_plus(psf, 8, 2, cols, w.h, RHO0, 8, tol=tol)
    assert C.info["kind"] == 2 and C.info["r"] == a.shape[0]
    v = synth.smoothed_normal_vectors(51, 2, w.nz, w.nx, 1.5)
    got = C.apply(torch.tensor(v, dtype=torch.float32, device="cuda")).cpu().numpy()
    want = DO.lr_apply(a, b, f32(v).astype(np.float64))
    for j in range(2):
        assert rel(got[j], want[j]) < 1e-4, (tol, j, rel(got[j], want[j]))
    # the symbol factors themselves: equal up to phases of the basis
    ga, gb = (x.cpu().numpy().astype(np.complex128) for x in C.symbol())
    for i in range(a.shape[0]):
        assert abs(np.linalg.norm(gb[i]) - 1.0) < 1e-5                       # orthonormal basis rows
        ph = np.vdot(b[i], gb[i]) / abs(np.vdot(b[i], gb[i]))
        if C.info["r"] <= 4:                                                   # well-separated directions
            assert rel(gb[i], b[i] * ph) < 1e-3, i
    C.close()


def test_psfplus_arguments_are_validated(built):
    w, P, m, A, D = built
    lib = _lib.load()
    out = ctypes.c_void_p(1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hv_approx_build_psfplus(D._a, A._a, ctypes.c_double(1e-3), ctypes.byref(out), stream) == _lib.HV_EINVAL
    assert out.value is None
    assert lib.hv_approx_build_psfplus(A._a, D._a, ctypes.c_double(0.0), ctypes.byref(out), stream) == _lib.HV_EINVAL
    w2 = ragged_workload(nz=30, nx=71, nb=6, nt=50, ns=2, nr=5)
    P2 = Problem.from_workload(w2)
    D2 = P2.approx_build_pdo(torch.tensor(w2.m, dtype=torch.float32, device="cuda"), RHO0, 8, ckpt=HV_CKPT_ALL)
    assert lib.hv_approx_build_psfplus(A._a, D2._a, ctypes.c_double(1e-3), ctypes.byref(out), stream) == _lib.HV_EINVAL
    assert "grids" in lib.hv_last_error().decode()
    D2.close()
