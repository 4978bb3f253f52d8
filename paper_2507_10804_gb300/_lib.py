"""ctypes binding of libhv (argument marshalling only; every step runs in the library).

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2507_10804_gb300.build``); loading fails loudly otherwise.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

c_int, c_double, c_size_t, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
ip = ctypes.POINTER(c_int)
fp = ctypes.c_void_p        # device float* / double* passed as integers
HEADER = os.path.join(_build.INCLUDE, "hv.h")

HV_OK, HV_EINVAL, HV_ENOMEM, HV_ECUDA, HV_ETIMEOUT, HV_EBUSY, HV_ENOTSUP = range(7)
HV_CKPT_ALL = -1
HV_OP_FWD, HV_OP_BORN, HV_OP_MIGRATE, HV_OP_GRAD, HV_OP_HV, HV_OP_WAVEFIELD, HV_OP_MISFIT, HV_OP_MISFITS = range(8)
HV_K_FWD, HV_K_ADVANCE, HV_K_ADJ, HV_K_OTHER = range(4)
HV_K_COUNT = 4
HV_LAUNCH_PLAIN, HV_LAUNCH_PDL, HV_LAUNCH_DATAFLOW = range(3)
HV_IMAGE_PAIRS, HV_IMAGE_FP64 = 0, 1


class HvGrid(ctypes.Structure):
    _fields_ = [("nz", c_int), ("nx", c_int), ("nb", c_int), ("h", c_double)]


class HvAcq(ctypes.Structure):
    _fields_ = [("ns", c_int), ("src_iz", ip), ("src_ix", ip), ("nr", c_int), ("rec_iz", ip), ("rec_ix", ip),
                ("nt", c_int), ("dt", c_double), ("f0", c_double), ("t0", c_double), ("vmax", c_double),
                ("R", c_double), ("sigma", c_double)]


class HvRequest(ctypes.Structure):
    _fields_ = [("kind", c_int), ("problem", c_void_p), ("m", fp), ("v", fp), ("k", c_int), ("d_obs", fp),
                ("out", fp), ("phi", fp), ("ckpt", c_int), ("approx", c_void_p), ("approx_mode", c_int)]


class HvRequestInfo(ctypes.Structure):
    _fields_ = [("kind", c_int), ("status", c_int), ("t_submit", c_double), ("t_start", c_double),
                ("t_done", c_double), ("ws_bytes", c_size_t), ("batch", c_int)]


class HvBatch(ctypes.Structure):
    _fields_ = [("n_hv", c_int), ("v", ctypes.POINTER(c_void_p)), ("k", ctypes.POINTER(c_int)),
                ("Hv", ctypes.POINTER(c_void_p)), ("n_grad", c_int), ("grad_dobs", ctypes.POINTER(c_void_p)),
                ("grad_phi", ctypes.POINTER(c_void_p)), ("grad", ctypes.POINTER(c_void_p)), ("n_misfit", c_int),
                ("misfit_dobs", ctypes.POINTER(c_void_p)), ("misfit_phi", ctypes.POINTER(c_void_p))]


HV_OP_FN = ctypes.CFUNCTYPE(c_int, c_void_p, fp, c_int, fp, c_void_p)


class HvOperator(ctypes.Structure):
    _fields_ = [("nz", c_int), ("nx", c_int), ("h", c_double), ("apply", HV_OP_FN), ("ctx", c_void_p)]


HV_QUAD_HD, HV_QUAD_A, HV_QUAD_AT, HV_QUAD_HD_RAW = 0, 1, 2, 3
HV_REQ_HV, HV_REQ_GRAD, HV_REQ_MISFIT, HV_REQ_APPROX = 0, 1, 2, 3
HV_APPROX_H, HV_APPROX_SQRT, HV_APPROX_INVSQRT, HV_APPROX_SQRT_T = 0, 1, 2, 3
HV_REQ_QUEUED, HV_REQ_RUNNING = 100, 101

_SIGS = {
    "hv_last_error": ([], ctypes.c_char_p),
    "hv_version": ([], c_int),
    "hv_create": ([ctypes.POINTER(HvGrid), ctypes.POINTER(HvAcq), ctypes.POINTER(c_void_p)], c_int),
    "hv_destroy": ([c_void_p], c_int),
    "hv_workspace_size": ([c_void_p, c_int, c_int, c_int, ctypes.POINTER(c_size_t)], c_int),
    "hv_fwd_model": ([c_void_p, fp, fp, fp, c_size_t, c_void_p], c_int),
    "hv_wavefield": ([c_void_p, fp, c_int, ip, fp, fp, c_size_t, c_void_p], c_int),
    "hv_born": ([c_void_p, fp, fp, c_int, fp, fp, c_size_t, c_void_p], c_int),
    "hv_migrate": ([c_void_p, fp, fp, fp, c_int, fp, c_size_t, c_void_p], c_int),
    "hv_misfit_grad": ([c_void_p, fp, fp, fp, fp, c_int, fp, c_size_t, c_void_p], c_int),
    "hv_hessian_apply": ([c_void_p, fp, fp, c_int, fp, c_int, fp, c_size_t, c_void_p], c_int),
    "hv_hessian_apply_f64out": ([c_void_p, fp, fp, c_int, fp, c_int, fp, c_size_t, c_void_p], c_int),
    "hv_hessian_apply_partial": ([c_void_p, fp, fp, c_int, fp, c_int, fp, c_size_t, c_void_p], c_int),
    "hv_image_fold": ([c_void_p, fp, c_int, fp, fp, c_void_p], c_int),
    "hv_hessian_apply_static": ([ctypes.POINTER(HvGrid), ctypes.POINTER(HvAcq), fp, fp, c_int, fp, c_int,
                                 c_void_p], c_int),
    "hv_status": ([c_void_p, ctypes.POINTER(c_int)], c_int),
    "hv_static_status": ([ctypes.POINTER(c_int)], c_int),
    "hv_set_wait_limit": ([c_void_p, c_double], c_int),
    "hv_inject_wait_timeout": ([c_void_p], c_int),
    "hv_misfit": ([c_void_p, fp, fp, fp, fp, c_size_t, c_void_p], c_int),
    "hv_misfit_models": ([c_void_p, c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                          fp, c_size_t, c_void_p], c_int),
    "hv_engine_workspace_size": ([c_void_p, c_int, ctypes.POINTER(c_size_t)], c_int),
    "hv_engine_create": ([c_void_p, c_int, fp, c_size_t, ctypes.POINTER(c_void_p)], c_int),
    "hv_engine_join": ([c_void_p, fp, fp, fp, c_void_p, ip], c_int),
    "hv_engine_tick": ([c_void_p, c_void_p, ip, ip], c_int),
    "hv_engine_active": ([c_void_p, ip], c_int),
    "hv_engine_destroy": ([c_void_p], c_int),
    "hv_engine_post": ([c_void_p, fp, fp, fp, c_void_p, ip], c_int),
    "hv_engine_serve": ([c_void_p, c_void_p], c_int),
    "hv_engine_poll": ([c_void_p, ip, ip, ip], c_int),
    "hv_engine_stop": ([c_void_p], c_int),
    "hv_server_set_engine": ([c_void_p, c_int], c_int),
    "hv_server_set_engine_loop": ([c_void_p, c_int], c_int),
    "hv_count_nonfinite": ([fp, c_size_t, fp, c_void_p], c_int),
    "hv_server_create": ([c_size_t, c_int, ctypes.POINTER(c_void_p)], c_int),
    "hv_server_destroy": ([c_void_p, c_double], c_int),
    "hv_submit": ([c_void_p, ctypes.POINTER(HvRequest), ctypes.POINTER(ctypes.c_ulonglong)], c_int),
    "hv_poll": ([c_void_p, ctypes.c_ulonglong, ctypes.POINTER(c_int)], c_int),
    "hv_wait": ([c_void_p, ctypes.c_ulonglong, c_double, ctypes.POINTER(c_int)], c_int),
    "hv_request_get_info": ([c_void_p, ctypes.c_ulonglong, ctypes.POINTER(HvRequestInfo)], c_int),
    "hv_server_set_batching": ([c_void_p, c_int], c_int),
    "hv_batch_workspace_size": ([c_void_p, ctypes.POINTER(HvBatch), c_int, ctypes.POINTER(c_size_t)], c_int),
    "hv_apply_batch": ([c_void_p, fp, ctypes.POINTER(HvBatch), c_int, fp, c_size_t, c_void_p], c_int),
    "hv_approx_psf_workspace_size": ([c_void_p, c_int, c_int, ctypes.POINTER(c_size_t)], c_int),
    "hv_approx_build_psf": ([c_void_p, fp, c_int, c_int, c_int, ctypes.POINTER(c_void_p), fp, c_size_t, c_void_p],
                            c_int),
    "hv_approx_info": ([c_void_p, ip], c_int),
    "hv_approx_psfs": ([c_void_p, fp, c_void_p], c_int),
    "hv_approx_pdo_workspace_size": ([c_void_p, c_int, ctypes.POINTER(c_size_t)], c_int),
    "hv_approx_build_pdo": ([c_void_p, fp, c_double, c_int, c_int, ctypes.POINTER(c_void_p), fp, c_size_t, c_void_p],
                            c_int),
    "hv_approx_pdo_symbol": ([c_void_p, fp, fp, c_void_p], c_int),
    "hv_approx_build_psfplus": ([c_void_p, c_void_p, c_double, ctypes.POINTER(c_void_p), c_void_p], c_int),
    "hv_approx_build_psfplus_sqrt": ([c_void_p, c_void_p, c_double, ctypes.POINTER(c_void_p), c_void_p], c_int),
    "hv_approx_sqrt_pdo": ([c_void_p, ctypes.POINTER(c_void_p), c_void_p], c_int),
    "hv_util_hermitian_eig": ([c_int, ctypes.POINTER(c_double), ctypes.POINTER(c_double), ctypes.POINTER(c_double)],
                              c_int),
    "hv_prior_apply": ([c_int, c_int, c_double, c_double, c_double, fp, c_int, fp, c_int, c_void_p], c_int),
    "hv_approx_lr_workspace_size": ([c_void_p, c_int, c_int, ctypes.POINTER(c_size_t)], c_int),
    "hv_approx_build_lr": ([c_void_p, fp, c_double, c_double, c_int, fp, c_int, c_int, ctypes.POINTER(c_void_p), fp,
                            c_size_t, c_void_p], c_int),
    "hv_approx_lr_eigs": ([c_void_p, ctypes.POINTER(c_double), fp, c_void_p], c_int),
    "hv_approx_apply": ([c_void_p, fp, c_int, fp, c_int, c_void_p], c_int),
    "hv_approx_build_psf_op": ([ctypes.POINTER(HvOperator), c_int, c_int, ctypes.POINTER(c_void_p), c_void_p], c_int),
    "hv_approx_build_pdo_op": ([ctypes.POINTER(HvOperator), c_double, c_int, ctypes.POINTER(c_void_p), c_void_p],
                               c_int),
    "hv_approx_build_lr_op": ([ctypes.POINTER(HvOperator), c_double, c_double, c_int, fp, c_int,
                               ctypes.POINTER(c_void_p), c_void_p], c_int),
    "hv_highpass_apply": ([c_int, c_int, c_double, c_double, fp, c_int, fp, c_void_p], c_int),
    "hv_set_highpass": ([c_void_p, c_double], c_int),
    "hv_filtered_create": ([ctypes.POINTER(HvOperator), c_double, c_int, ctypes.POINTER(c_void_p)], c_int),
    "hv_filtered_operator": ([c_void_p, ctypes.POINTER(HvOperator)], c_int),
    "hv_filtered_destroy": ([c_void_p], c_int),
    "hv_quad_create": ([c_int, c_int, c_double, c_double, c_int, c_int, ctypes.POINTER(c_double), c_double, c_double,
                        ctypes.POINTER(c_void_p)], c_int),
    "hv_quad_apply": ([c_void_p, c_int, fp, c_int, fp, c_void_p], c_int),
    "hv_quad_objective": ([c_void_p, fp, fp, c_int, c_int, fp, fp, c_void_p], c_int),
    "hv_quad_tables": ([c_void_p, fp, fp, fp, fp, c_void_p], c_int),
    "hv_quad_operator": ([c_void_p, ctypes.POINTER(HvOperator)], c_int),
    "hv_quad_destroy": ([c_void_p], c_int),
    "hv_approx_destroy": ([c_void_p], c_int),
    "hv_posterior_create": ([c_int, c_int, c_double, c_double, c_double, c_void_p, c_int, ctypes.POINTER(c_void_p)],
                            c_int),
    "hv_posterior_solve": ([c_void_p, ctypes.POINTER(HvOperator), fp, c_int, fp, c_double, c_int, ip, c_void_p],
                           c_int),
    "hv_posterior_apply": ([c_void_p, fp, c_int, fp, c_void_p], c_int),
    "hv_posterior_sample": ([c_void_p, fp, fp, c_int, fp, c_double, c_int, ip, c_void_p], c_int),
    "hv_posterior_correct": ([c_void_p, ctypes.POINTER(HvOperator), fp, c_int, c_int, c_double, c_int, c_void_p],
                             c_int),
    "hv_posterior_eigs": ([c_void_p, ctypes.POINTER(c_double), fp, c_void_p], c_int),
    "hv_posterior_rank": ([c_void_p], c_int),
    "hv_posterior_destroy": ([c_void_p], c_int),
    "hv_gpcn_propose": ([c_int, c_int, fp, fp, fp, c_double, fp, fp, c_void_p], c_int),
    "hv_gpcn_accept": ([c_int, c_int, fp, fp, fp, fp, fp, fp, fp, fp, c_void_p], c_int),
    "hv_tile_menu_size": ([], c_int),
    "hv_set_launch_mode": ([c_void_p, c_int], c_int),
    "hv_set_step_fusion": ([c_void_p, c_int], c_int),
    "hv_set_fused_transforms": ([c_int], c_int),
    "hv_set_resident": ([c_void_p, c_int], c_int),
    "hv_set_image_precision": ([c_void_p, c_int], c_int),
    "hv_resident_fits": ([c_void_p], c_int),
    "hv_tile_menu": ([c_int, ip, ip], c_int),
    "hv_tile_menu_info": ([c_int, ip], c_int),
    "hv_autotune": ([c_void_p, c_int, fp, c_size_t, c_void_p, ip, ctypes.POINTER(ctypes.c_float)], c_int),
    "hv_set_tiles": ([c_void_p, ip], c_int),
    "hv_get_tiles": ([c_void_p, ip], c_int),
    "hv_set_graphs": ([c_void_p, c_int], c_int),
    "hv_profile": ([c_void_p, c_int], c_int),
    "hv_profile_read": ([c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(c_double)], c_int),
    "hv_kernel_launches": ([], ctypes.c_longlong),
    "hv_checkpoint_schedule": ([c_int, c_int, ip, c_int, ip, ctypes.POINTER(ctypes.c_longlong)], c_int),
}

_lib = None


def header_symbols() -> list[str]:
    """Every function the public header declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?\s*\*?\s*\b(hv_\w+)\s*\(", text, flags=re.M)))


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libhv.so is not built ({_build.LIB}); run __graft_entry__.build() first")
        lib = ctypes.CDLL(_build.LIB)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


class HvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libhv error {code}: {msg}")
        self.code = code


def check(rc: int) -> None:
    if rc != HV_OK:
        raise HvError(rc, load().hv_last_error().decode())
