"""PDO probing approximation on the GPU (hv_approx_build_pdo / hv_approx_apply)
against the FP64 oracle (oracle/pdo_oracle.py): the spectral separation of the
GPU's own H v_p, the frequency weights, the low-rank-symbol apply on identical
(a, b), and the whole build against the oracle's."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import pdo_oracle as DO
from paper_2507_10804_gb300 import _lib, synth
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem
from tests._helpers import f32, oracle_problem, ragged_workload, rel

pytestmark = pytest.mark.gpu
RHO0 = 0.15          # rad/m on the 10 m grid (Nyquist 0.314)


@pytest.fixture(scope="module")
def ragged():
    w = ragged_workload(nz=37, nx=71, nb=6, nt=150, ns=3, nr=7)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    return w, P, m


@pytest.mark.parametrize("r,ckpt", [(8, HV_CKPT_ALL), (4, 6), (16, HV_CKPT_ALL)])
def test_pdo_columns_and_weights_match_oracle_on_the_same_hessian(ragged, r, ckpt):
    w, P, m = ragged
    A = P.approx_build_pdo(m, RHO0, r, ckpt=ckpt)
    assert A.info["kind"] == 1 and A.info["r"] == r
    a, b = A.symbol()
    a, b = a.cpu().numpy().astype(np.complex128), b.cpu().numpy().astype(np.complex128)
    vp = torch.tensor(DO.probe(w.nz, w.nx, w.h, RHO0, r)[None], dtype=torch.float32, device="cuda")
    Hvp = P.hessian_apply(m, vp, ckpt=ckpt).cpu().numpy().astype(np.float64)[0]
    want_a = DO.extract_columns(Hvp, w.h, RHO0, r)
    want_b = DO.frequency_weights(w.nz, w.nx, w.h, RHO0, r)
    for k in range(r):
        assert rel(a[k], want_a[k]) < 1e-5, (k, rel(a[k], want_a[k]))
    assert np.abs(b - want_b).max() < 1e-5 * np.abs(want_b).max()
    A.close()


def test_pdo_apply_matches_oracle_on_the_same_symbol(ragged):
    w, P, m = ragged
    A = P.approx_build_pdo(m, RHO0, 8, ckpt=6)
    a, b = A.symbol()
    a, b = a.cpu().numpy().astype(np.complex128), b.cpu().numpy().astype(np.complex128)
    v = synth.smoothed_normal_vectors(31, 3, w.nz, w.nx, 1.5)
    got = A.apply(torch.tensor(v, dtype=torch.float32, device="cuda")).cpu().numpy()
    want = DO.lr_apply(a, b, f32(v).astype(np.float64))
    for j in range(3):
        assert rel(got[j], want[j]) < 1e-5, (j, rel(got[j], want[j]))
    A.close()


def test_pdo_build_matches_oracle_build(ragged):
    w, P, m = ragged
    A = P.approx_build_pdo(m, RHO0, 8, ckpt=HV_CKPT_ALL)
    a, b = A.symbol()
    a = a.cpu().numpy().astype(np.complex128)
    want_a, want_b = DO.build(lambda V: O.hessian_apply(oracle_problem(w), f32(w.m), V), w.nz, w.nx, w.h, RHO0, 8)
    assert rel(a, want_a) < 2e-4, rel(a, want_a)
    v = synth.smoothed_normal_vectors(41, 1, w.nz, w.nx, 1.5)
    got = A.apply(torch.tensor(v, dtype=torch.float32, device="cuda")).cpu().numpy()[0]
    want = DO.lr_apply(want_a, want_b, f32(v).astype(np.float64))[0]
    assert rel(got, want) < 2e-4, rel(got, want)
    A.close()


def test_pdo_arguments_are_validated(ragged):
    w, P, m = ragged
    lib = _lib.load()
    out = ctypes.c_void_p()
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.hv_approx_build_pdo(P._h, m.data_ptr(), ctypes.c_double(RHO0), 7, 5, ctypes.byref(out), ws.data_ptr(),
                                   ws.numel(), stream) == _lib.HV_EINVAL            # odd r
    assert lib.hv_approx_build_pdo(P._h, m.data_ptr(), ctypes.c_double(0.3), 8, 5, ctypes.byref(out), ws.data_ptr(),
                                   ws.numel(), stream) == _lib.HV_EINVAL            # window reaches Nyquist
    assert "Nyquist" in lib.hv_last_error().decode()
    assert lib.hv_approx_build_pdo(P._h, m.data_ptr(), ctypes.c_double(RHO0), 8, 5, ctypes.byref(out), ws.data_ptr(),
                                   1024, stream) == _lib.HV_ENOMEM
    assert out.value is None
    A = P.approx_build_pdo(m, RHO0, 8, ckpt=5)
    v = torch.zeros((1, w.nz, w.nx), dtype=torch.float32, device="cuda")
    o = torch.empty_like(v)
    assert lib.hv_approx_apply(A._a, v.data_ptr(), 1, o.data_ptr(), 1, stream) == _lib.HV_ENOTSUP
    assert lib.hv_approx_psfs(A._a, o.data_ptr(), stream) == _lib.HV_EINVAL
    A.close()
