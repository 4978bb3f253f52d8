"""The Matern prior's operators on the GPU (hv_prior_apply, section 2.1) against
the FP64 oracle (oracle/lowrank_oracle.py): A^-1 and R^-1 run the fast DCT of
csrc/hv_dct.cu (one real 2D DFT of the reordered field), on even, odd,
non-square and one-row or one-column grids, and for more fields than one
transform batch holds."""
import numpy as np
import pytest
import torch

from oracle import lowrank_oracle as LO
from paper_2507_10804_gb300 import synth
from paper_2507_10804_gb300.hv import prior_apply
from tests._helpers import f32, rel

pytestmark = pytest.mark.gpu
H, DELTA, GAMMA = 10.0, 1.0, 2500.0


@pytest.mark.parametrize("nz,nx,k", [(1, 1, 2), (1, 7, 3), (9, 1, 3), (5, 8, 2), (16, 16, 3), (37, 71, 2),
                                     (64, 64, 70), (48, 70, 1)])
def test_inverse_prior_matches_oracle(nz, nx, k):
    v = synth.normal(nz * 31 + nx + k, k * nz * nx).reshape(k, nz, nx)
    vt = torch.tensor(v, dtype=torch.float32, device="cuda")
    for op, fn, tol in ((1, LO.prior_Ainv, 1e-5), (3, LO.prior_Rinv, 2e-5), (0, LO.prior_A, 1e-5),
                        (2, LO.prior_R, 2e-5)):
        got = prior_apply(vt, H, DELTA, GAMMA, op).cpu().numpy()
        for j in range(k):
            want = fn(f32(v[j]), H, DELTA, GAMMA)
            assert rel(got[j], want) < tol, (op, j, rel(got[j], want))


def test_inverse_prior_inverts_the_stencil():
    nz, nx, k = 40, 56, 4
    v = torch.tensor(synth.normal(3, k * nz * nx).reshape(k, nz, nx), dtype=torch.float32, device="cuda")
    back = prior_apply(prior_apply(v, H, DELTA, GAMMA, 0), H, DELTA, GAMMA, 1)
    assert rel(back.cpu().numpy(), v.cpu().numpy()) < 1e-5
