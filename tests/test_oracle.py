"""Pins of the FP64 CPU oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: a closed
form (the 2D Green's function of eq. (pde), polynomial exactness of the
8th-order Laplacian, the Ricker wavelet's zeros), an exact identity
(adjointness, energy conservation of the undamped leapfrog, Hessian symmetry),
finite differences of the forward map and of the misfit (eq. (grad)), or a
dense Hessian assembled column by column (the 2 N N_s solves of section 3).
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2507_10804_gb300 import synth


def small_problem(nz=12, nx=14, nb=5, h=10.0, nt=60, ns=2, nr=5, f0=20.0, seed=11, sigma=1.0):
    m = synth.gradient_grf_model(seed, nz, nx, h, 1500.0, 2200.0, std=60.0, corr_len=30.0)
    vmax = float(m.max())
    dt = synth.cfl_dt(h, vmax, 0.45)
    acq = synth.surface_acquisition(nx, ns, nr, src_iz=1, rec_iz=0)
    P = O.Problem(nz=nz, nx=nx, nb=nb, h=h, nt=nt, dt=dt, f0=f0, t0=1.5 / f0, vmax=vmax,
                  src_iz=acq.src_iz, src_ix=acq.src_ix, rec_iz=acq.rec_iz, rec_ix=acq.rec_ix,
                  sigma=sigma)
    return P, m


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# --------------------------------------------------------------------------- stencil
def test_laplacian_exact_on_degree9_polynomials():
    """An 8th-order central second derivative is exact for degree <= 9 and not for 10."""
    P = O.Problem(nz=30, nx=30, nb=0, h=0.5, nt=1, dt=1e-3, f0=10, t0=0.15, vmax=1.0,
                  src_iz=[0], src_ix=[0], rec_iz=[[0]], rec_ix=[[0]])
    z = (np.arange(30) - 14.5)[:, None] * P.h * np.ones((1, 30))
    x = (np.arange(30) - 14.5)[None, :] * P.h * np.ones((30, 1))
    inner = (slice(4, 26), slice(4, 26))
    rng = np.random.default_rng(0)
    a = rng.standard_normal(10)
    b = rng.standard_normal(10)
    u = sum(a[p] * x ** p + b[p] * z ** p for p in range(10))
    exact = sum(a[p] * p * (p - 1) * x ** (p - 2) + b[p] * p * (p - 1) * z ** (p - 2) for p in range(2, 10))
    Lu = O.laplacian(P, u)
    assert rel(Lu[inner], exact[inner]) < 1e-11
    # degree 10: the truncation error is the constant c h^8 10!, c != 0
    err10 = O.laplacian(P, x ** 10)[inner] - (90 * x ** 8)[inner]
    assert np.all(np.abs(err10) > 1.0) and np.ptp(err10) < 1e-6 * np.abs(err10).max()


def test_laplacian_symmetric_with_dirichlet_ghosts():
    P, _ = small_problem()
    rng = np.random.default_rng(1)
    u = rng.standard_normal((P.NZ, P.NX))
    w = rng.standard_normal((P.NZ, P.NX))
    a = np.vdot(O.laplacian(P, u), w)
    b = np.vdot(u, O.laplacian(P, w))
    assert abs(a - b) < 1e-12 * abs(a)


# --------------------------------------------------------------------------- source / sponge / E
def test_ricker_closed_form_features():
    f0, dt = 12.0, 1e-4
    t0 = 1.5 / f0
    nt = int(4 * t0 / dt)
    s = O.ricker(nt, dt, f0, t0)
    n0 = int(round(t0 / dt))
    assert abs(s[n0] - 1.0) < 1e-12                          # peak value 1 at t0
    tz = 1.0 / (np.sqrt(2.0) * np.pi * f0)                    # zero crossings at t0 +- tz
    i = int(np.floor((t0 + tz) / dt))
    assert s[i] > 0 > s[i + 1] or s[i] < 0 < s[i + 1]
    # amplitude spectrum |S(f)| ~ f^2 exp(-f^2/f0^2) peaks at f0
    spec = np.abs(np.fft.rfft(np.concatenate([s, np.zeros(20 * nt)])))
    freqs = np.fft.rfftfreq(21 * nt, dt)
    assert abs(freqs[np.argmax(spec)] - f0) < 0.05 * f0


def test_sponge_rate_profile():
    P, _ = small_problem(nb=6)
    q = O.sponge_q(P)
    L = P.nb * P.h
    qmax = 3 * P.vmax * np.log(1 / P.R) / (2 * L)
    assert np.all(q[P.nb:P.nb + P.nz, P.nb:P.nb + P.nx] == 0.0)
    assert abs(q[0, P.NX // 2] - qmax) < 1e-12 * qmax
    assert abs(q[P.nb - 1, P.NX // 2] - qmax / P.nb ** 2) < 1e-12 * qmax
    col = q[:P.nb, P.NX // 2]
    assert np.all(np.diff(col) < 0)


def test_extension_fold_adjoint_and_constants():
    P, _ = small_problem()
    rng = np.random.default_rng(2)
    x = rng.standard_normal((P.nz, P.nx))
    y = rng.standard_normal((P.NZ, P.NX))
    assert abs(np.vdot(O.extend(P, x), y) - np.vdot(x, O.fold(P, y))) < 1e-12 * np.abs(x).sum()
    assert np.all(O.extend(P, np.full((P.nz, P.nx), 3.5)) == 3.5)
    ones = O.fold(P, np.ones((P.NZ, P.NX)))
    assert ones[0, 0] == (P.nb + 1) ** 2 and ones[P.nz // 2, P.nx // 2] == 1.0
    assert ones[0, P.nx // 2] == P.nb + 1


# --------------------------------------------------------------------------- forward
def _green_conv(r, t, c, f0, t0):
    """u = (1/2 pi) int_0^inf s(t - (r/c) cosh phi) dphi: the 2D Green's function
    H(t - r/c) / (2 pi sqrt(t^2 - r^2/c^2)) of (1/c^2) d_tt - lap, convolved with s."""
    def s(tt):
        a = (np.pi * f0 * (tt - t0)) ** 2
        return (1 - 2 * a) * np.exp(-a)
    if t < r / c + t0 - 0.25:
        return 0.0
    phimax = np.arccosh(max(1.0, (t + 1.0) / (r / c)))
    val, _ = integrate.quad(lambda ph: s(t - (r / c) * np.cosh(ph)), 0.0, phimax, limit=400)
    return val / (2 * np.pi)


def test_forward_matches_2d_greens_function():
    c, h, n, nb, f0 = 2000.0, 5.0, 200, 30, 10.0
    t0 = 1.5 / f0
    dt = 0.4 * h / c
    nt = int(0.36 / dt)
    rz = np.array([[100, 100, 140, 128]])
    rx = np.array([[120, 140, 100, 128]])
    P = O.Problem(nz=n, nx=n, nb=nb, h=h, nt=nt, dt=dt, f0=f0, t0=t0, vmax=c,
                  src_iz=[100], src_ix=[100], rec_iz=rz, rec_ix=rx)
    d = O.fwd_model(P, np.full((n, n), c))
    tt = (np.arange(nt) + 1) * dt             # d[n] samples u^{n+1} = u((n+1) dt)
    for i in range(rz.shape[1]):
        r = h * np.hypot(rz[0, i] - 100, rx[0, i] - 100)
        w = tt < r / c + t0 + 0.1
        exact = np.array([_green_conv(r, t, c, f0, t0) for t in tt[w]])
        num = d[0, w, i]
        assert rel(num, exact) < 1e-2, (r, rel(num, exact))
        # a one-step time shift or a wrong delta scaling would fail the bound
        assert rel(np.concatenate([[0.0], num[:-1]]), exact) > 2e-2


def test_undamped_leapfrog_conserves_discrete_energy():
    """With no sponge, E^{n+1/2} = |(u^{n+1}-u^n)/dt|^2_{1/m^2} - <u^{n+1}, L u^n> is constant
    once the source has died out (L symmetric, so the leapfrog is symplectic)."""
    P, m = small_problem(nz=24, nx=24, nb=0, nt=260, ns=1)
    U = O.wavefield(P, m, 0)
    w = 1.0 / m ** 2
    def energy(n):   # uses u^{n+1} = U[n], u^{n+2} = U[n+1]
        du = (U[n + 1] - U[n]) / P.dt
        return np.sum(w * du * du) - np.sum(U[n + 1] * O.laplacian(P, U[n]))
    n_quiet = int(3.2 * P.t0 / P.dt)
    e = np.array([energy(n) for n in range(n_quiet, P.nt - 1, 7)])
    assert e.min() > 0
    assert (e.max() - e.min()) / e.max() < 1e-10


def test_sponge_absorbs():
    P, m = small_problem(nz=40, nx=40, nb=20, nt=900, ns=1, f0=25.0)
    U = O.wavefield(P, m, 0)
    en = np.sum(U ** 2, axis=(1, 2))
    assert en[-1] < 1e-4 * en.max()


# --------------------------------------------------------------------------- adjoints
def test_dot_test_S_inverse():
    P, m = small_problem(nt=40)
    rng = np.random.default_rng(3)
    F = rng.standard_normal((P.nt, P.NZ, P.NX))
    G = rng.standard_normal((P.nt, P.NZ, P.NX))
    a = np.vdot(O.solve_S(P, m, F), G)
    b = np.vdot(F, O.solve_ST(P, m, G))
    assert abs(a - b) <= 1e-12 * abs(a)


def test_dot_test_born_migration():
    P, m = small_problem()
    rng = np.random.default_rng(4)
    dm = rng.standard_normal((P.nz, P.nx))
    r = rng.standard_normal((P.ns, P.nt, P.nr))
    a = np.vdot(O.born(P, m, dm)[0], r)
    b = np.vdot(dm, O.adjoint(P, m, r))
    assert abs(a - b) <= 1e-12 * abs(a)


# --------------------------------------------------------------------------- derivatives
def test_born_is_derivative_of_forward_map():
    P, m = small_problem(nt=80)
    dm = synth.smoothed_normal_vectors(5, 1, P.nz, P.nx, 1.5)[0] * 20.0
    J = O.born(P, m, dm)[0]
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        fd = (O.fwd_model(P, m + eps * dm) - O.fwd_model(P, m - eps * dm)) / (2 * eps)
        errs.append(rel(fd, J))
    assert errs[-1] < 1e-5
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0   # O(eps^2)


def test_gradient_matches_finite_differences():
    P, m = small_problem(nt=80)
    dobs = O.fwd_model(P, synth.perturbed_model(m, P.h, 6, amp=0.03, radius=40.0))
    phi, g = O.misfit_grad(P, m, dobs)
    p = synth.smoothed_normal_vectors(7, 1, P.nz, P.nx, 1.5)[0] * 10.0
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        fp, _ = O.misfit_grad(P, m + eps * p, dobs)
        fm, _ = O.misfit_grad(P, m - eps * p, dobs)
        errs.append(abs((fp - fm) / (2 * eps) - np.vdot(g, p)) / abs(np.vdot(g, p)))
    assert phi > 0
    assert errs[-1] < 1e-5
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_hessian_equals_gradient_difference_at_zero_residual():
    """At d_obs = f(m) the full and Gauss-Newton Hessians coincide, so the central
    difference of the gradient along v converges to H_GN v (O(eps^2))."""
    P, m = small_problem(nt=80, sigma=0.5)
    dobs = O.fwd_model(P, m)
    v = synth.smoothed_normal_vectors(8, 1, P.nz, P.nx, 1.5)[0] * 10.0
    Hv = O.hessian_apply(P, m, v)
    errs = []
    for eps in (1.0, 0.5, 0.25):      # perturbations of a few m/s: above the FP64 floor
        gp = O.misfit_grad(P, m + eps * v, dobs)[1]
        gm = O.misfit_grad(P, m - eps * v, dobs)[1]
        errs.append(rel((gp - gm) / (2 * eps), Hv))
    assert errs[-1] < 1e-6
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_hessian_symmetric_positive_semidefinite():
    P, m = small_problem()
    rng = np.random.default_rng(9)
    u = rng.standard_normal((P.nz, P.nx))
    v = rng.standard_normal((P.nz, P.nx))
    Hu, Hv = O.hessian_apply(P, m, np.stack([u, v]))
    a, b = np.vdot(u, Hv), np.vdot(Hu, v)
    assert abs(a - b) <= 1e-12 * abs(a)
    assert np.vdot(v, Hv) > 0 and np.vdot(u, Hu) > 0


def test_dense_hessian_bruteforce_8x8():
    """F assembled column by column from N Born solves, H = F^T F / sigma^2 by a dense
    product, against the adjoint-based Hessian apply on every unit vector."""
    P, m = small_problem(nz=8, nx=8, nb=8, nt=200, ns=2, nr=4, sigma=0.7)
    N = P.nz * P.nx
    E = np.eye(N).reshape(N, P.nz, P.nx)
    J = O.born(P, m, E).reshape(N, -1).T          # [ns*nt*nr, N]
    H_dense = J.T @ J / P.sigma ** 2
    H_apply = O.hessian_apply(P, m, E).reshape(N, N).T
    assert rel(H_apply, H_dense) < 1e-12
    assert np.allclose(H_dense, H_dense.T, rtol=0, atol=1e-12 * np.abs(H_dense).max())
    assert np.linalg.eigvalsh(H_dense).min() > -1e-10 * np.abs(H_dense).max()


def test_extended_image_folds_to_the_hessian_and_adds_over_shots():
    """The extended image before the fold (the per-source sum of section 3): its fold is the
    Hessian apply; <E u, ext> is the Born-data inner product <F u, F v> / sigma^2 (no adjoint
    solve on that side); the images of two shot blocks add up to the image of all shots."""
    P, m = small_problem(ns=3, sigma=0.8)
    u, v = synth.smoothed_normal_vectors(12, 2, P.nz, P.nx, 1.5)
    ext = O.hessian_image(P, m, v)[0]
    assert np.array_equal(O.fold(P, ext), O.hessian_apply(P, m, v))
    Fu, Fv = O.born(P, m, u[None])[0], O.born(P, m, v[None])[0]
    a, b = np.vdot(O.extend(P, u), ext), np.vdot(Fu, Fv) / P.sigma ** 2
    assert abs(a - b) <= 1e-12 * abs(b)
    parts = []
    for idx in ([0, 2], [1]):
        Q = O.Problem(nz=P.nz, nx=P.nx, nb=P.nb, h=P.h, nt=P.nt, dt=P.dt, f0=P.f0, t0=P.t0, vmax=P.vmax,
                      src_iz=np.asarray(P.src_iz)[idx], src_ix=np.asarray(P.src_ix)[idx],
                      rec_iz=np.asarray(P.rec_iz)[idx], rec_ix=np.asarray(P.rec_ix)[idx], sigma=P.sigma)
        parts.append(O.hessian_image(Q, m, v)[0])
    assert rel(parts[0] + parts[1], ext) < 1e-13


def test_multithreaded_oracle_is_deterministic():
    P, m = small_problem(ns=4)
    v = synth.smoothed_normal_vectors(10, 1, P.nz, P.nx, 1.5)
    a = O.hessian_apply(P, m, v, nthreads=1)
    b = O.hessian_apply(P, m, v, nthreads=4)
    assert np.array_equal(a, b)
