"""The high-pass filter before the PSF and PDO approximations (sections 3.2 and
3.7) on the GPU against the FP64 oracle (oracle/highpass_oracle.py): the
filter itself, PSF and PDO builds of the filtered quadratic-model Hessian
F_hp H_d F_hp against the oracle builds of the oracle's own filtered Hessian,
and the approximation quality on the wave-equation Hessian with and without
the filter."""
import numpy as np
import pytest
import torch

from oracle import highpass_oracle as HP
from oracle import pdo_oracle as DO
from oracle import psf_oracle as PO
from oracle import quadratic_oracle as QO
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import (HV_CKPT_ALL, Filtered, Problem, Quad, approx_build_pdo_op, approx_build_psf_op,
                                      highpass_apply)
from tests._helpers import f32, rel

pytestmark = pytest.mark.gpu
NZ, NX, H = 48, 70, 10.0
LAM = [40.0, 30.0, 20.0, 12.0, 8.0, 5.0]
DELTA, GAMMA = 1.0, 2500.0


@pytest.mark.parametrize("nz,nx,k", [(48, 70, 3), (37, 71, 5), (64, 64, 70)])
def test_filter_matches_oracle(nz, nx, k):
    v = synth.normal(5 + k, k * nz * nx).reshape(k, nz, nx)
    got = highpass_apply(torch.tensor(v, dtype=torch.float32, device="cuda"), 8.0, 0.04).cpu().numpy()
    want = HP.highpass(f32(v), 8.0, 0.04)
    for j in range(k):
        assert rel(got[j], want[j]) < 2e-6, (j, rel(got[j], want[j]))


def test_filtered_quadratic_builds_match_oracle():
    Q = Quad(NZ, NX, H, LAM, DELTA, GAMMA, taper=5)
    q = QO.make(NZ, NX, H, LAM, L=5)
    rc = 0.05
    F = Filtered(Q, rc, max_k=4)
    hd_f = HP.filtered_operator(lambda V: QO.apply_Hd(q, V), H, rc)
    A = approx_build_psf_op(F, 8, 4)
    got = A.psfs().cpu().numpy()
    want = PO.build(hd_f, NZ, NX, 8, 2)
    assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()
    rho0 = 0.12
    D = approx_build_pdo_op(F, rho0, 8)
    a = D.symbol()[0].cpu().numpy().astype(np.complex128)
    want_a = DO.extract_columns(hd_f(DO.probe(NZ, NX, H, rho0, 8)[None])[0], H, rho0, 8)
    for k in range(8):
        assert rel(a[k], want_a[k]) < 1e-4, (k, rel(a[k], want_a[k]))
    A.close()
    D.close()
    F.close()


@pytest.mark.parametrize("S,B", [(8, 2), (12, 1)])
def test_filtered_handle_build_windows_are_the_filtered_hessian(S, B):
    """hv_set_highpass: the PSF build applies F_hp H_d F_hp to the impulse batches; its windows are exact
    copies of the filter, the Hessian apply and the filter composed through the public calls."""
    w = synth.workload(3, nt=300, ns=4)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    rc = 2 * np.pi * (0.5 * w.f0) / float(w.m.max())
    P.set_highpass(rc)
    A = P.approx_build_psf(m, S, B * B, ckpt=6)
    V = torch.tensor(PO.impulse_batches(w.nz, w.nx, S, B), dtype=torch.float32, device="cuda")
    Hv = highpass_apply(P.hessian_apply(m, highpass_apply(V, w.h, rc), ckpt=6), w.h, rc).cpu().numpy()
    assert np.array_equal(A.psfs().cpu().numpy(), PO.extract(Hv.astype(np.float64), S, B).astype(np.float32))
    # the filtered operator's outputs have no mean (phi(0) = 0 on the output side)
    assert np.abs(Hv.reshape(B * B, -1).sum(axis=1)).max() < 1e-4 * np.abs(Hv).sum() / (B * B)
    A.close()


def test_psf_approximation_quality_with_and_without_the_filter_is_reported():
    """Not a parity bar: on the 64 x 64 (+20 sponge) model with 8 surface shots the wave-equation Hessian is
    far from local, so PSF windows of radius 7 cells capture little of it with or without the filter (relative
    error about 0.93 either way; the filtered operator's impulse responses also carry the filter's own spread)."""
    w = synth.workload(3, nt=500, ns=8)
    P = Problem.from_workload(w)
    m = torch.tensor(w.m, dtype=torch.float32, device="cuda")
    v = torch.tensor(synth.smoothed_normal_vectors(23, 3, w.nz, w.nx, 1.0), dtype=torch.float32, device="cuda")
    rc = 2 * np.pi * (0.5 * w.f0) / float(w.m.max())                # cutoff at half the peak frequency
    res = {}
    for name, cut in (("H_d", 0.0), ("F H_d F", rc)):
        P.set_highpass(cut)
        A = P.approx_build_psf(m, 8, 4, ckpt=HV_CKPT_ALL)
        approx = A.apply(v).cpu().numpy()
        if cut > 0:
            exact = highpass_apply(P.hessian_apply(m, highpass_apply(v, w.h, cut), ckpt=HV_CKPT_ALL), w.h, cut)
        else:
            exact = P.hessian_apply(m, v, ckpt=HV_CKPT_ALL)
        exact = exact.cpu().numpy()
        assert np.isfinite(approx).all()
        res[name] = float(np.mean([rel(approx[j], exact[j]) for j in range(3)]))
        A.close()
    print(f"PSF approximation (8-cell lattice, R = 7) relative error: H_d {res['H_d']:.3f}, "
          f"F H_d F (rho_c = {rc:.4f} rad/m) {res['F H_d F']:.3f}")
    assert res["H_d"] < 1.0 and res["F H_d F"] < 1.0
