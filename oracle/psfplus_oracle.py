"""FP64 oracle of the PSF+ low-rank symbol (paper section 3.6).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

What it computes, in the paper's order:

1. Symbol rows from the PSFs (section 3.5): s(x_k, xi) = sum_d p_k(d) e^{i xi . d},
   the conjugated DFT of the PSF placed at the origin of the grid; with the
   interpolation weights W the PSF method's symbol is S_psf = W S[I_r, :].
2. The SVD S[I_r, :] = U Sigma V^H keeps the dominant r' right singular
   vectors as the basis B = V^H[:r'] of the symbol's frequency dependence, so
   S_psf = A0 B with A0 = W U[:, :r'] Sigma[:r'].
3. A is refined against the PDO symbol columns S~[:, I_c] (section 3.4):
       min_A ||A B[:, I_c] - S~[:, I_c]||_F^2 + alpha ||A - A0||_F^2,
       alpha = ||B[:, I_c]||_F^2 / ||B||_F^2,
   whose minimiser is A = (S~_c B_c^H + alpha A0)(B_c B_c^H + alpha I)^{-1}.
The approximation is applied as sum_i D_{A[:, i]} F^-1 D_{B[i]} F (eq. (lr-psido)).

With spd = True (section 3.7) the rows and columns are those of the square
root, sqrt(max(Re s, 0)), and the result B is applied as B B^T.

Readings (stated in the design notes): r' = the number of singular values at
least tol * sigma_1 (tol = 1e-3), at most 32; the PSF weights are those of the
PSF oracle (bilinear on the lattice); the DFT is the periodic transform of the
interior grid, as for the PDO columns.

Pins: tests/test_psfplus_oracle.py.
"""
from __future__ import annotations

import numpy as np

from oracle import pdo_oracle as DO
from oracle import psf_oracle as PO

MAX_RANK = 32


def psf_rows(P: np.ndarray, nz: int, nx: int) -> np.ndarray:
    """[r, nz, nx] complex symbol rows s(x_k, xi) = sum_d p_k(d) exp(i xi . d) on the DFT grid."""
    r, W, _ = P.shape
    R = (W - 1) // 2
    if W > nz or W > nx:
        raise ValueError("PSF window larger than the grid")
    E = np.zeros((r, nz, nx))
    for dz in range(-R, R + 1):
        for dx in range(-R, R + 1):
            E[:, dz % nz, dx % nx] = P[:, dz + R, dx + R]
    return np.conj(np.fft.fft2(E))


def rank_of(sv: np.ndarray, tol: float = 1e-3) -> int:
    return int(min(MAX_RANK, max(1, np.count_nonzero(sv >= tol * sv[0]))))


def psf_plus(P: np.ndarray, S: int, B: int, cols: np.ndarray, h: float, rho0: float, r_c: int, tol: float = 1e-3,
             spd: bool = False):
    """(a [r', nz, nx], b [r', nz, nx]) of the PSF+ symbol from PSFs P (lattice S, batches B x B) and
    PDO columns cols [r_c, nz, nx] at the snapped samples of (rho0, r_c).  spd: the symbol of the
    square root (section 3.7): rows and columns replaced by sqrt(max(Re s, 0)) before the SVD."""
    _, nz, nx = cols.shape
    N = nz * nx
    rows = psf_rows(P, nz, nx).reshape(P.shape[0], N)
    if spd:
        rows = np.sqrt(np.maximum(rows.real, 0.0)).astype(np.complex128)
        cols = np.sqrt(np.maximum(cols.real, 0.0)).astype(np.complex128)
    Wt = PO.weights(nz, nx, S).reshape(P.shape[0], N).T            # N x r
    U, sv, Vh = np.linalg.svd(rows, full_matrices=False)
    rr = rank_of(sv, tol)
    Bm = Vh[:rr]                                                     # r' x N
    A0 = Wt @ (U[:, :rr] * sv[:rr])                                   # N x r'
    idx, _, _ = DO.samples(nz, nx, h, rho0, r_c)
    Ic = (idx[:, 0] % nz) * nx + (idx[:, 1] % nx)
    Bc = Bm[:, Ic]                                                   # r' x r_c
    Sc = cols.reshape(r_c, N).T                                      # N x r_c
    alpha = np.linalg.norm(Bc) ** 2 / np.linalg.norm(Bm) ** 2
    M = Bc @ Bc.conj().T + alpha * np.eye(rr)
    A = np.linalg.solve(M.T, (Sc @ Bc.conj().T + alpha * A0).T).T    # (Sc Bc^H + alpha A0) M^-1
    return A.T.reshape(rr, nz, nx), Bm.reshape(rr, nz, nx), alpha, A0.T.reshape(rr, nz, nx)
