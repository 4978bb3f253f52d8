"""The fused low-rank-symbol transforms (hv_lrfft.cu: the library's own 2D DFTs
with the symbol products fused in, used on power-of-two grids) against the FP64
oracle and against the cuFFT path, for every length split the kernels have
(16 ... 512 points per axis), through the quadratic test model's operator A and
through a PDO approximation built from wave-equation H v."""
import numpy as np
import pytest
import torch

from oracle import pdo_oracle as DO
from oracle import quadratic_oracle as QO
from oracle import spd_oracle as SO
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300._lib import (HV_APPROX_H, HV_APPROX_SQRT, HV_APPROX_SQRT_T, HV_QUAD_A, HV_QUAD_AT,
                                         HV_QUAD_HD_RAW)
from paper_2507_10804_gb300.hv import HV_CKPT_ALL, Problem, Quad, set_fused_transforms
from tests._helpers import f32, ragged_workload, rel

pytestmark = pytest.mark.gpu
H = 10.0
LAM = [40.0, 30.0, 20.0, 12.0]
DELTA, GAMMA = 1.0, 2500.0
# (nz, nx): together the lengths 16, 32, 64, 128, 256 and 512 on both axes
GRIDS = [(16, 512), (512, 16), (32, 128), (64, 64), (256, 256)]


@pytest.fixture(autouse=True)
def _fused_default():
    set_fused_transforms(True)
    yield
    set_fused_transforms(True)


def _vecs(seed, k, nz, nx):
    v = synth.smoothed_normal_vectors(seed, k, nz, nx, 1.5)
    return f32(v).astype(np.float64), torch.tensor(v, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("nz,nx", GRIDS)
def test_quadratic_operator_matches_oracle(nz, nx):
    taper = max(1, min(nz, nx) // 8)
    Q = Quad(nz, nx, H, LAM, DELTA, GAMMA, taper=taper)
    q = QO.make(nz, nx, H, LAM, L=taper)
    for op, fn in ((HV_QUAD_A, QO.apply_A), (HV_QUAD_AT, QO.apply_AT), (HV_QUAD_HD_RAW, QO.apply_Hd_raw)):
        v, vt = _vecs(300 + op, 3, nz, nx)
        got = Q.apply(vt, op).cpu().numpy()
        want = fn(q, v)
        for j in range(3):
            assert rel(got[j], want[j]) < 2e-5, (nz, nx, op, j, rel(got[j], want[j]))
    Q.close()


@pytest.mark.parametrize("nz,nx", [(64, 64), (256, 256), (16, 512)])
def test_fused_and_library_transforms_agree(nz, nx):
    taper = max(1, min(nz, nx) // 8)
    Qf = Quad(nz, nx, H, LAM, DELTA, GAMMA, taper=taper)
    set_fused_transforms(False)
    Qc = Quad(nz, nx, H, LAM, DELTA, GAMMA, taper=taper)
    set_fused_transforms(True)
    # 70 vectors: more than one apply batch of the library path at 256 x 256
    _, vt = _vecs(310, 70, nz, nx)
    for op in (HV_QUAD_A, HV_QUAD_AT, HV_QUAD_HD_RAW):
        a, b = Qf.apply(vt, op).cpu().numpy(), Qc.apply(vt, op).cpu().numpy()
        for j in (0, 33, 69):
            assert rel(a[j], b[j]) < 2e-6, (nz, nx, op, j, rel(a[j], b[j]))
    Qf.close()
    Qc.close()


def test_pdo_on_a_power_of_two_grid():
    w = ragged_workload(nz=32, nx=64, nb=6, nt=150, ns=3, nr=7)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    rho0 = 0.15
    D = P.approx_build_pdo(m, rho0, 8, ckpt=HV_CKPT_ALL)
    Q = D.sqrt()
    set_fused_transforms(False)
    Dc = P.approx_build_pdo(m, rho0, 8, ckpt=HV_CKPT_ALL)
    Qc = Dc.sqrt()
    set_fused_transforms(True)
    v, vt = _vecs(320, 3, w.nz, w.nx)
    a, b = (x.cpu().numpy().astype(np.complex128) for x in D.symbol())
    got = D.apply(vt).cpu().numpy()
    want = DO.lr_apply(a, b, v)
    for j in range(3):
        assert rel(got[j], want[j]) < 1e-5, (j, rel(got[j], want[j]))
    assert rel(got, Dc.apply(vt).cpu().numpy()) < 2e-6
    qa, qb = (x.cpu().numpy().astype(np.complex128) for x in Q.symbol())
    for mode, want in ((HV_APPROX_SQRT, DO.lr_apply(qa, qb, v)), (HV_APPROX_SQRT_T, SO.lr_apply_T(qa, qb, v)),
                       (HV_APPROX_H, SO.spd_apply(qa, qb, v))):
        got = Q.apply(vt, mode).cpu().numpy()
        for j in range(3):
            assert rel(got[j], want[j]) < 1e-5, (mode, j, rel(got[j], want[j]))
        assert rel(got, Qc.apply(vt, mode).cpu().numpy()) < 2e-6, mode
    for x in (Q, Qc, D, Dc):
        x.close()
