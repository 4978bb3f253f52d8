"""Pins of the gpCN oracle (oracle/gpcn_oracle.py):

* with the exact Laplace approximation of a Gaussian posterior Delta is constant,
  so every proposal is accepted (section 2.3);
* the proposal preserves N(m_map, H~^-1): the covariance of m' - m_map is the
  same as that of m - m_map for any beta;
* with an inexact H~ the chain still samples the posterior: the mean and
  covariance of a long chain on a 3-dimensional Gaussian match it, and the
  reversed acceptance rule does not.
"""
import numpy as np

from oracle import gpcn_oracle as GO

MU = np.array([1.0, -2.0, 0.5])
A_ = np.array([[2.0, 0.3, 0.0], [0.3, 1.0, 0.2], [0.0, 0.2, 0.5]])
HP = A_ @ A_.T + 0.2 * np.eye(3)                      # posterior precision
COV = np.linalg.inv(HP)


def phi(m):
    d = m - MU
    return 0.5 * d @ HP @ d + 3.0


def _normals(seed, n, cov):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, 3)) @ np.linalg.cholesky(cov).T, rng.uniform(size=n)


def test_exact_laplace_accepts_everything():
    zetas, us = _normals(1, 500, COV)
    us = np.minimum(us, 1 - 1e-12)
    _, acc = GO.chain(np.zeros(3), MU, 0.7, phi, lambda d: HP @ d, zetas, us)
    assert acc.all()


def test_proposal_preserves_the_gaussian():
    for beta in (0.1, 0.5, 0.95):
        # Cov(m' - map) = (1 - beta^2) C + beta^2 C for independent m - map, zeta ~ N(0, C)
        I = np.eye(3)
        lin = np.sqrt(1 - beta ** 2) * I
        np.testing.assert_allclose(lin @ COV @ lin.T + beta ** 2 * COV, COV, atol=1e-15)
        np.testing.assert_allclose(GO.propose(MU + 1.0, MU, beta, np.zeros(3)) - MU,
                                   np.sqrt(1 - beta ** 2) * np.ones(3), atol=1e-15)


def _run(accept_rule, n=60000):
    Ht = 0.6 * HP + 0.3 * np.diag(np.diag(HP))                  # an inexact approximation
    zetas, us = _normals(3, n, np.linalg.inv(Ht))
    orig = GO.accept
    GO.accept = accept_rule
    try:
        S, acc = GO.chain(MU.copy(), MU, 0.5, phi, lambda d: Ht @ d, zetas, us)
    finally:
        GO.accept = orig
    return S[2000:], acc


def test_inexact_laplace_chain_samples_the_posterior():
    S, acc = _run(GO.accept)
    assert 0.2 < acc.mean() < 0.999
    np.testing.assert_allclose(S.mean(axis=0), MU, atol=0.05)
    np.testing.assert_allclose(np.cov(S.T), COV, atol=0.08 * np.abs(COV).max())
    # planted mistake: accept iff log u < Delta(m') - Delta(m_k)
    S2, _ = _run(lambda dc, dn, u: bool(np.log(u) < dn - dc))
    assert np.abs(np.cov(S2.T) - COV).max() > 0.15 * np.abs(COV).max()
