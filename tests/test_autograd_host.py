"""The autograd wrapper's plumbing, on the CPU with a stand-in problem whose
forward map is a dense linear map A (so F = A and F* = A^T exactly)."""
import torch

from paper_2507_10804_gb300.autograd import fwd_model, misfit


class LinearProblem:
    sigma = 0.5

    def __init__(self, nz=3, nx=4, ns=2, nt=5, nr=3, seed=0):
        g = torch.Generator().manual_seed(seed)
        self.shape_m, self.shape_d = (nz, nx), (ns, nt, nr)
        self.A = torch.randn(ns * nt * nr, nz * nx, generator=g, dtype=torch.float64)

    def fwd_model(self, m):
        return (self.A @ m.reshape(-1).to(torch.float64)).reshape(self.shape_d).to(m.dtype)

    def migrate(self, m, r, ckpt=-1):
        return (self.A.T @ r.reshape(-1).to(torch.float64)).reshape(self.shape_m).to(m.dtype)

    def misfit_grad(self, m, d_obs, ckpt=-1):
        r = self.fwd_model(m).to(torch.float64) - d_obs.to(torch.float64)
        phi = 0.5 * (r * r).sum() / self.sigma ** 2
        return phi, self.migrate(m, (r / self.sigma ** 2).to(m.dtype))

    def misfit(self, m, d_obs):
        return self.misfit_grad(m, d_obs)[0]

    def born(self, m, dm):
        return (self.A @ dm.reshape(dm.shape[0], -1).T.to(torch.float64)).T.reshape(dm.shape[0], *self.shape_d)


def test_backward_is_migration_and_gradcheck():
    P = LinearProblem()
    m = torch.randn(P.shape_m, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: fwd_model(P, x), (m,))
    dobs = torch.randn(P.shape_d, dtype=torch.float64)
    phi = misfit(P, m, dobs)
    phi.backward()
    r = (P.A @ m.detach().reshape(-1) - dobs.reshape(-1)) / P.sigma ** 2
    assert torch.allclose(m.grad.reshape(-1), P.A.T @ r)
    # the chain rule scales by the incoming gradient; no gradient wanted: the misfit alone
    m.grad = None
    (3.0 * misfit(P, m, dobs)).backward()
    assert torch.allclose(m.grad.reshape(-1), 3.0 * (P.A.T @ r))
    with torch.no_grad():
        assert torch.allclose(misfit(P, m, dobs), 0.5 * (r * r).sum() * P.sigma ** 2)


def test_forward_mode_is_born():
    P = LinearProblem()
    m = torch.randn(P.shape_m, dtype=torch.float64)
    dm = torch.randn(P.shape_m, dtype=torch.float64)
    import torch.autograd.forward_ad as fwAD
    with fwAD.dual_level():
        d = fwd_model(P, fwAD.make_dual(m, dm))
        tangent = fwAD.unpack_dual(d).tangent
    assert torch.allclose(tangent.reshape(-1), P.A @ dm.reshape(-1))
