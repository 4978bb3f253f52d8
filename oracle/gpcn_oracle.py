"""FP64 oracle of the generalized preconditioned Crank-Nicolson (gpCN) step
(paper section 2.3).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

What it computes (eq. (gpcn) and the acceptance rule after it):
* proposal m' = m_map + sqrt(1 - beta^2) (m_k - m_map) + beta zeta, zeta ~ N(0, Gamma~_post);
* Delta(m) = Phi(m) - 1/2 (m - m_map)^T H~ (m - m_map), H~ = Gamma~_post^-1;
* accept with probability min(1, exp(Delta(m_k) - Delta(m'))): given u ~ U(0, 1),
  accept iff log u < Delta(m_k) - Delta(m').

Pins: tests/test_gpcn_oracle.py.
"""
from __future__ import annotations

import numpy as np


def propose(m, m_map, beta: float, zeta):
    return m_map + np.sqrt(1.0 - beta * beta) * (m - m_map) + beta * zeta


def delta(phi: float, m, m_map, Ht_apply) -> float:
    d = np.asarray(m, dtype=np.float64) - m_map
    return float(phi - 0.5 * np.vdot(d, Ht_apply(d)))


def accept(delta_cur: float, delta_new: float, u: float) -> bool:
    return bool(np.log(u) < delta_cur - delta_new)


def chain(m0, m_map, beta, phi, Ht_apply, zetas, us):
    """Run len(us) gpCN steps; returns (samples [n, ...], accepted [n])."""
    m = np.asarray(m0, dtype=np.float64)
    dcur = delta(phi(m), m, m_map, Ht_apply)
    out, acc = [], []
    for zeta, u in zip(zetas, us):
        mp = propose(m, m_map, beta, zeta)
        dnew = delta(phi(mp), mp, m_map, Ht_apply)
        ok = accept(dcur, dnew, u)
        if ok:
            m, dcur = mp, dnew
        out.append(m)
        acc.append(ok)
    return np.stack(out), np.array(acc)
