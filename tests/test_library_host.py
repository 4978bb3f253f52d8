"""Host-side checks of libhv that need no GPU: exported symbols, the checkpoint
schedule (valid and optimal), and argument validation in hv_create."""
import ctypes

import numpy as np
import pytest

from oracle import revolve_dp as R
from paper_2507_10804_gb300 import _lib
from paper_2507_10804_gb300.hv import checkpoint_schedule


@pytest.fixture(scope="module")
def lib():
    from paper_2507_10804_gb300 import build
    build.build()
    return _lib.load()


def test_library_exports_every_header_symbol(lib):
    names = _lib.header_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert lib.hv_version() >= 100


def test_fused_transform_switch_is_host_only(lib):
    """The process-wide default for new approximations is set without touching a GPU."""
    assert lib.hv_set_fused_transforms(0) == 0
    assert lib.hv_set_fused_transforms(1) == 0


def simulate(actions, nt, slots):
    """Replay a schedule: every adjoint step exactly once in reverse order, each
    with u^n available; snapshot slots within budget and never clobbered while in use."""
    j = 0
    where = ("zero", "zero")          # buffers holding (cur, prev)
    slot_state = {}
    adj = []
    adv = 0
    seen_forward = 0
    for op, a0, a1 in actions:
        if op == 0:
            assert a0 == j == seen_forward
            seen_forward += 1
            j += 1
            where = ("work", where[0])
        elif op == 1:
            assert 0 <= a0 < slots and a1 == j
            if where != (("slotA", a0), ("slotB", a0)):
                assert where[0] != ("slotB", a0) and where[1] != ("slotA", a0)
            slot_state[a0] = j
            where = (("slotA", a0), ("slotB", a0))
        elif op == 2:
            if a0 < 0:
                j, where = 0, ("zero", "zero")
            else:
                assert slot_state.get(a0) == a1
                j, where = a1, (("slotA", a0), ("slotB", a0))
        elif op == 3:
            assert a0 == j
            j += 1
            adv += 1
            where = ("work", where[0])
        elif op == 4:
            assert j in (a0, a0 + 1), (a0, j)
            adj.append(a0)
        else:
            raise AssertionError(op)
    assert seen_forward == nt
    assert adj == list(range(nt - 1, -1, -1))
    return adv


@pytest.mark.parametrize("nt,slots", [(1, 1), (2, 1), (7, 1), (12, 2), (40, 3), (97, 4), (150, 5), (64, 63)])
def test_schedule_valid_and_optimal(lib, nt, slots):
    acts, adv = checkpoint_schedule(nt, slots)
    assert simulate(acts.tolist(), nt, slots) == adv
    assert adv == R.min_advances_dp(nt, slots)


def test_schedule_matches_exhaustive_search_on_tiny_chains(lib):
    for s in (1, 2):
        for nt in range(1, 9):
            assert checkpoint_schedule(nt, s)[1] == R.min_advances_bruteforce(nt, s)


def test_schedule_cost_at_paper_scale(lib):
    # 3000 steps with 30 snapshots per shot (the 384 x 1152 workload)
    acts, adv = checkpoint_schedule(3000, 30)
    assert simulate(acts.tolist(), 3000, 30) == adv
    assert adv < 2 * 3000


def _create(lib, nz=8, nx=8, nb=2, ns=1, nr=2, src=((0, 3),), recs=((0, 1), (0, 5)), nt=10, dt=1e-3,
            vmax=2000.0, R=1e-3, sigma=1.0):
    g = _lib.HvGrid(nz, nx, nb, 10.0)
    si = np.array([s[0] for s in src], np.int32)
    sx = np.array([s[1] for s in src], np.int32)
    ri = np.array([r[0] for r in recs], np.int32)
    rx = np.array([r[1] for r in recs], np.int32)
    a = _lib.HvAcq(ns, si.ctypes.data_as(_lib.ip), sx.ctypes.data_as(_lib.ip), nr, ri.ctypes.data_as(_lib.ip),
                   rx.ctypes.data_as(_lib.ip), nt, dt, 15.0, 0.1, vmax, R, sigma)
    h = ctypes.c_void_p()
    rc = lib.hv_create(ctypes.byref(g), ctypes.byref(a), ctypes.byref(h))
    return rc, lib.hv_last_error().decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(src=((0, 8),)), "source node"),
    (dict(recs=((0, 1), (9, 5))), "receiver 1"),
    (dict(recs=((0, 1), (0, 1))), "duplicates"),
    (dict(dt=0.0), "must be > 0"),
    (dict(R=1.5), "reflection"),
    (dict(nz=0), "grid"),
    (dict(nt=0), "nt = 0"),
])
def test_create_rejects_bad_arguments_before_touching_the_gpu(lib, kw, needle):
    rc, msg = _create(lib, **kw)
    assert rc == _lib.HV_EINVAL
    assert needle in msg


def test_approximation_entry_points_validate_before_touching_the_gpu(lib):
    out = ctypes.c_void_p(1)
    assert lib.hv_approx_build_psf(None, None, 12, 4, 8, ctypes.byref(out), None, 0, None) == _lib.HV_EINVAL
    assert out.value is None
    assert "null" in lib.hv_last_error().decode()
    out = ctypes.c_void_p(1)
    assert lib.hv_approx_build_pdo(None, None, ctypes.c_double(0.01), 8, 8, ctypes.byref(out), None, 0, None) \
        == _lib.HV_EINVAL
    assert out.value is None
    assert lib.hv_approx_apply(None, None, 1, None, 0, None) == _lib.HV_EINVAL
    n = ctypes.c_size_t()
    assert lib.hv_approx_psf_workspace_size(None, 4, 8, ctypes.byref(n)) == _lib.HV_EINVAL
    info = (ctypes.c_int * 11)()
    assert lib.hv_approx_info(None, info) == _lib.HV_EINVAL
    assert lib.hv_approx_destroy(None) == _lib.HV_OK


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (5, 2), (40, 3), (64, 4)])
def test_hermitian_eigensolver(n, seed):
    """The host Jacobi routine behind the PSF+ build: A V = V diag(w), V unitary, w descending,
    against numpy's eigh on random Hermitian matrices (with a repeated eigenvalue for n >= 5)."""
    from paper_2507_10804_gb300.hv import hermitian_eig
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = X @ X.conj().T
    if n >= 5:
        Q, _ = np.linalg.qr(X)
        d = np.sort(rng.standard_normal(n))[::-1]
        d[1] = d[2]
        A = (Q * d) @ Q.conj().T
    w, V = hermitian_eig(A)
    assert np.all(np.diff(w) <= 1e-12 * max(1.0, abs(w).max()))
    np.testing.assert_allclose(w, np.sort(np.linalg.eigvalsh(A))[::-1], atol=1e-10 * max(1.0, abs(w).max()))
    np.testing.assert_allclose(V.conj().T @ V, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(A @ V, V * w, atol=1e-10 * max(1.0, abs(w).max()))


def test_hermitian_eigensolver_rejects_non_hermitian(lib):
    A = np.array([[1.0, 2.0], [0.0, 1.0]], dtype=np.complex128)
    w, V = np.empty(2), np.empty((2, 2), dtype=np.complex128)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.hv_util_hermitian_eig(2, A.view(np.float64).ctypes.data_as(dp), w.ctypes.data_as(dp),
                                   V.view(np.float64).ctypes.data_as(dp))
    assert rc == _lib.HV_EINVAL and "Hermitian" in lib.hv_last_error().decode()


def test_new_entry_points_validate_before_touching_a_gpu(lib):
    """Null handles, empty batches and bad limits are rejected with HV_EINVAL on the host."""
    E = _lib.HV_EINVAL
    assert lib.hv_set_wait_limit(None, 1.0) == E
    assert lib.hv_inject_wait_timeout(None) == E
    assert lib.hv_set_image_precision(None, _lib.HV_IMAGE_FP64) == E
    assert lib.hv_set_highpass(None, 0.1) == E
    assert lib.hv_static_status(None) == E
    assert lib.hv_server_set_batching(None, 8) == E
    assert lib.hv_filtered_create(None, 0.1, 4, ctypes.byref(ctypes.c_void_p())) == E
    assert lib.hv_filtered_operator(None, None) == E
    assert lib.hv_filtered_destroy(None) == 0
    assert lib.hv_highpass_apply(8, 8, 10.0, 0.1, None, 1, None, None) == E
    assert lib.hv_image_fold(None, None, 1, None, None, None) == E
    b = _lib.HvBatch()                                   # no entries at all
    n = ctypes.c_size_t()
    assert lib.hv_batch_workspace_size(None, ctypes.byref(b), -1, ctypes.byref(n)) == E
    assert "batch" in lib.hv_last_error().decode() or "handle" in lib.hv_last_error().decode()
    assert lib.hv_hessian_apply_partial(None, None, None, 1, None, -1, None, 0, None) == E
    arr = (ctypes.c_void_p * 2)(1, 2)                    # non-null entries: nothing is dereferenced before the checks
    assert lib.hv_misfit_models(None, 0, arr, arr, arr, None, 0, None) == E
    assert "models" in lib.hv_last_error().decode()
    assert lib.hv_misfit_models(None, 2, None, arr, arr, None, 0, None) == E
    holes = (ctypes.c_void_p * 2)(1, None)
    assert lib.hv_misfit_models(None, 2, arr, holes, arr, None, 0, None) == E
    assert "model 1" in lib.hv_last_error().decode()
    assert lib.hv_misfit_models(None, 2, arr, arr, arr, None, 0, None) == E
    assert "handle" in lib.hv_last_error().decode()
    cnt = ctypes.c_ulonglong()
    assert lib.hv_count_nonfinite(None, 4, ctypes.byref(cnt), None) == E
    assert lib.hv_count_nonfinite(None, 0, None, None) == E
    # the misfit engine and its device-resident loop, and the server's lane switches
    i1, i2, i3 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.hv_engine_create(None, 4, None, 0, ctypes.byref(ctypes.c_void_p())) == E
    assert lib.hv_engine_create(None, 0, None, 0, ctypes.byref(ctypes.c_void_p())) == E
    assert lib.hv_engine_join(None, None, None, None, None, ctypes.byref(i1)) == E
    assert lib.hv_engine_tick(None, None, ctypes.byref(i1), ctypes.byref(i2)) == E
    assert lib.hv_engine_post(None, None, None, None, None, ctypes.byref(i1)) == E
    assert lib.hv_engine_serve(None, None) == E
    assert lib.hv_engine_poll(None, ctypes.byref(i1), ctypes.byref(i2), ctypes.byref(i3)) == E
    assert lib.hv_engine_stop(None) == E
    assert lib.hv_engine_active(None, ctypes.byref(i1)) == E
    assert lib.hv_engine_destroy(None) == 0
    assert lib.hv_server_set_engine(None, 8) == E
    assert lib.hv_server_set_engine_loop(None, 1) == E
