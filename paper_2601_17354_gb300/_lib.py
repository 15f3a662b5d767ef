"""ctypes binding of libpocketgs.so (the C ABI declared in include/pocketgs.h).

Argument marshalling only: every step of the rasterizer runs in the library's CUDA kernels.
Loading fails loudly if the library cannot be built or found; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

PGS_OK = 0
PGS_ERR_INVALID_ARG = -1
PGS_ERR_NO_RENDER = -2
PGS_ERR_CAPACITY = -3
PGS_ERR_NONFINITE = -4
PGS_ERR_CUDA = -6
PGS_ERR_OOM = -7
PGS_ERR_INTERNAL = -8
PGS_ERR_TOO_LARGE = -9
PGS_ERR_NOT_PD = -10
PGS_ERR_TIMEOUT = -11

PGS_MVS_CENSUS_TARGET = 0
PGS_MVS_CENSUS_REFERENCE = 1
PGS_MVS_COST = 2
PGS_MVS_AGGREGATED = 3
PGS_MVS_PLANE_MAPS = 4

PGS_BUF_KEYS = 0
PGS_BUF_VALUES = 1
PGS_BUF_RANGES = 2
PGS_BUF_T_FINAL = 3
PGS_BUF_LAST = 4
PGS_BUF_GRAD2D = 5
PGS_BUF_TILES_TOUCHED = 6
PGS_BUF_NCOMP = 7

PGS_STAGES = ["project", "bin", "sort", "composite_fwd", "loss", "composite_bwd", "project_bwd",
              "adam", "project_bwd_adam"]

EXPORTED = ["pgs_create", "pgs_destroy", "pgs_reserve", "pgs_render", "pgs_render_l1", "pgs_loss_l1",
            "pgs_backward", "pgs_step", "pgs_status", "pgs_read_buffer", "pgs_strerror",
            "pgs_profile", "pgs_stage_times", "pgs_launch_count", "pgs_backward_step",
            "pgs_batch_create", "pgs_batch_destroy", "pgs_batch_step", "pgs_batch_capture",
            "pgs_batch_losses", "pgs_batch_status", "pgs_batch_launch_count", "pgs_set_variant",
            "pgs_batch_set_variant", "pgs_batch_time_variants", "pgs_time_variants",
            "pgs_set_variants", "pgs_time_variants_split",
            "pgs_init_create", "pgs_init_destroy", "pgs_knn", "pgs_features_init",
            "pgs_mlp_param_count", "pgs_mlp_pack", "pgs_mlp_forward", "pgs_mlp_grad", "pgs_mlp_adam",
            "pgs_apply_mlp", "pgs_make_targets", "pgs_batch_set_views", "pgs_batch_reserve",
            "pgs_batch_steps", "pgs_batch_time_render", "pgs_set_replay_cache", "pgs_loss_dssim",
            "pgs_ba_create", "pgs_ba_destroy", "pgs_ba_project", "pgs_ba_step", "pgs_ba_solve", "pgs_ba_stage_times",
            "pgs_mvs_create", "pgs_mvs_destroy", "pgs_mvs_depth_range", "pgs_mvs_select_reference",
            "pgs_mvs_depth", "pgs_mvs_read", "pgs_mvs_fuse", "pgs_mvs_stage_times",
            "pgs_trace_pixels", "pgs_sort_pairs_static_status", "pgs_render_batch", "pgs_backward_batch",
            "pgs_selftest_timeout"]

VARIANTS = [(p, d) for p in (1, 2, 4) for d in (64, 128, 256)]


class PgsCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("viewmat", C.c_float * 12),
                ("near_z", C.c_float), ("bg", C.c_float * 3)]


class PgsGaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("pad_", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class PgsRenderDesc(C.Structure):
    _fields_ = [("scene", C.c_int32), ("pad_", C.c_int32), ("cam", PgsCamera), ("image", C.c_void_p),
                ("target", C.c_void_p), ("dL_dimage", C.c_void_p)]


class PgsMlp(C.Structure):
    _fields_ = [("master", C.c_void_p), ("W1", C.c_void_p), ("W2", C.c_void_p), ("W3", C.c_void_p)]


class PgsConfig(C.Structure):
    _fields_ = [("tile", C.c_int32), ("reserved_", C.c_int32), ("pair_capacity", C.c_int64),
                ("adam_b1", C.c_float), ("adam_b2", C.c_float), ("adam_eps", C.c_float),
                ("lr", C.c_float * 6)]


class PgsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().pgs_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libpocketgs.so")


def lib():
    """Load libpocketgs.so, building it with nvcc first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            path = _build.build()
            L = C.CDLL(path)
            P, I, I64 = C.c_void_p, C.c_int, C.c_int64
            L.pgs_create.argtypes = [C.POINTER(P), C.POINTER(PgsConfig), P]
            L.pgs_create.restype = I
            L.pgs_destroy.argtypes = [P]
            L.pgs_destroy.restype = None
            L.pgs_reserve.argtypes = [P, I64, C.c_int32, C.c_int32, I64]
            L.pgs_reserve.restype = I
            L.pgs_render.argtypes = [P, C.POINTER(PgsGaussians), C.POINTER(PgsCamera), P]
            L.pgs_render.restype = I
            L.pgs_loss_l1.argtypes = [P, P, P, I64, P, P]
            L.pgs_loss_l1.restype = I
            L.pgs_render_l1.argtypes = [P, C.POINTER(PgsGaussians), C.POINTER(PgsCamera), P, P, P, P]
            L.pgs_render_l1.restype = I
            L.pgs_backward.argtypes = [P, P, C.POINTER(PgsGaussians)]
            L.pgs_backward.restype = I
            L.pgs_step.argtypes = [P] + [C.POINTER(PgsGaussians)] * 4 + [I64]
            L.pgs_backward_step.argtypes = [P, P] + [C.POINTER(PgsGaussians)] * 3 + [I64]
            L.pgs_backward_step.restype = I
            L.pgs_step.restype = I
            L.pgs_status.argtypes = [P, C.POINTER(I64)]
            L.pgs_status.restype = I
            L.pgs_read_buffer.argtypes = [P, I, P, I64, C.POINTER(I64)]
            L.pgs_read_buffer.restype = I
            L.pgs_trace_pixels.argtypes = [P, P, I64, C.c_int32, P, P, P, P, P, P]
            L.pgs_trace_pixels.restype = I
            L.pgs_profile.argtypes = [P, I]
            L.pgs_profile.restype = I
            L.pgs_stage_times.argtypes = [P, P, P]
            L.pgs_stage_times.restype = I
            L.pgs_launch_count.argtypes = [P]
            L.pgs_launch_count.restype = I64
            L.pgs_sort_pairs_static.argtypes = [P, P, P, P, I64, C.c_int32, P]
            L.pgs_sort_pairs_static.restype = I
            L.pgs_sort_pairs_static_status.argtypes = [P]
            L.pgs_sort_pairs_static_status.restype = I
            L.pgs_batch_create.argtypes = [C.POINTER(P), C.POINTER(PgsConfig), C.c_int32,
                                           C.POINTER(PgsGaussians), C.POINTER(PgsGaussians),
                                           C.POINTER(PgsGaussians), C.c_int32,
                                           C.POINTER(PgsRenderDesc), I64, P]
            L.pgs_batch_create.restype = I
            L.pgs_batch_destroy.argtypes = [P]
            L.pgs_batch_destroy.restype = None
            L.pgs_selftest_timeout.argtypes = [P]
            L.pgs_selftest_timeout.restype = I
            L.pgs_render_batch.argtypes = [P]
            L.pgs_render_batch.restype = I
            L.pgs_backward_batch.argtypes = [P, C.POINTER(PgsGaussians)]
            L.pgs_backward_batch.restype = I
            for name in ("pgs_batch_step", "pgs_batch_capture"):
                getattr(L, name).argtypes = [P]
                getattr(L, name).restype = I
            L.pgs_batch_set_views.argtypes = [P, C.POINTER(PgsCamera), C.POINTER(C.c_void_p)]
            L.pgs_batch_set_views.restype = I
            L.pgs_batch_reserve.argtypes = [P, C.c_int64]
            L.pgs_batch_reserve.restype = I
            L.pgs_batch_steps.argtypes = [P, C.POINTER(C.c_int64)]
            L.pgs_batch_steps.restype = I
            L.pgs_batch_time_render.argtypes = [P, I, C.POINTER(C.c_float)]
            L.pgs_batch_time_render.restype = I
            L.pgs_set_replay_cache.argtypes = [P, I]
            L.pgs_set_replay_cache.restype = I
            L.pgs_loss_dssim.argtypes = [P, P, P, I, I, C.c_float, P, P]
            L.pgs_loss_dssim.restype = I
            L.pgs_batch_losses.argtypes = [P, P]
            L.pgs_batch_losses.restype = I
            L.pgs_batch_status.argtypes = [P, C.POINTER(I64)]
            L.pgs_batch_status.restype = I
            L.pgs_batch_launch_count.argtypes = [P]
            L.pgs_batch_launch_count.restype = I64
            L.pgs_set_variant.argtypes = [P, C.c_int32, C.c_int32]
            L.pgs_set_variant.restype = I
            L.pgs_batch_set_variant.argtypes = [P, C.c_int32, C.c_int32]
            L.pgs_batch_set_variant.restype = I
            L.pgs_batch_time_variants.argtypes = [P, C.c_int32, P]
            L.pgs_batch_time_variants.restype = I
            L.pgs_time_variants.argtypes = [P, P, P, C.c_int32, P]
            L.pgs_time_variants.restype = I
            L.pgs_set_variants.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
            L.pgs_set_variants.restype = I
            L.pgs_time_variants_split.argtypes = [P, P, P, C.c_int32, P, P]
            L.pgs_time_variants_split.restype = I
            L.pgs_init_create.argtypes = [C.POINTER(P), P]
            L.pgs_init_create.restype = I
            L.pgs_init_destroy.argtypes = [P]
            L.pgs_init_destroy.restype = None
            L.pgs_knn.argtypes = [P, P, I64, C.c_int32, P]
            L.pgs_knn.restype = I
            L.pgs_features_init.argtypes = [P, P, I64, P, C.c_float, P, P, P, C.POINTER(PgsGaussians)]
            L.pgs_features_init.restype = I
            L.pgs_mlp_param_count.argtypes = []
            L.pgs_mlp_param_count.restype = I
            L.pgs_mlp_pack.argtypes = [P, C.POINTER(PgsMlp)]
            L.pgs_mlp_pack.restype = I
            L.pgs_mlp_forward.argtypes = [P, C.POINTER(PgsMlp), P, I64, P]
            L.pgs_mlp_forward.restype = I
            L.pgs_mlp_grad.argtypes = [P, C.POINTER(PgsMlp), P, P, I64, P, P]
            L.pgs_mlp_grad.restype = I
            L.pgs_mlp_adam.argtypes = [P, C.POINTER(PgsMlp), P, P, P, C.c_float, I64]
            L.pgs_mlp_adam.restype = I
            L.pgs_apply_mlp.argtypes = [P, P, C.POINTER(PgsGaussians), C.POINTER(PgsGaussians), P]
            L.pgs_apply_mlp.restype = I
            L.pgs_make_targets.argtypes = [P, C.POINTER(PgsGaussians), C.POINTER(PgsGaussians), P]
            L.pgs_make_targets.restype = I
            F, D = C.c_float, C.c_double
            L.pgs_ba_create.argtypes = [C.POINTER(P), C.c_int32, I64, I64, P]
            L.pgs_ba_create.restype = I
            L.pgs_ba_destroy.argtypes = [P]
            L.pgs_ba_destroy.restype = None
            L.pgs_ba_project.argtypes = [P, P, P, P, P, P, I64, C.POINTER(F), P, P]
            L.pgs_ba_project.restype = I
            L.pgs_ba_step.argtypes = [P, P, P, P, P, P, P, C.POINTER(F), F, F, F, P, P, C.POINTER(D)]
            L.pgs_ba_step.restype = I
            L.pgs_ba_solve.argtypes = [P, P, P, P, P, P, P, C.POINTER(F), F, F, C.c_int32, F,
                                       C.POINTER(D), C.POINTER(C.c_int32)]
            L.pgs_ba_solve.restype = I
            L.pgs_ba_stage_times.argtypes = [P, P, P, P, P, P, P, C.POINTER(F), F, F, F, P]
            L.pgs_ba_stage_times.restype = I
            CamP = C.POINTER(PgsCamera)
            L.pgs_mvs_create.argtypes = [C.POINTER(P), C.c_int32, C.c_int32, C.c_int32, P]
            L.pgs_mvs_create.restype = I
            L.pgs_mvs_destroy.argtypes = [P]
            L.pgs_mvs_destroy.restype = None
            L.pgs_mvs_depth_range.argtypes = [P, CamP, P, I64, C.POINTER(D)]
            L.pgs_mvs_depth_range.restype = I
            L.pgs_mvs_select_reference.argtypes = [P, CamP, C.c_int32, C.c_int32, D, C.POINTER(D),
                                                   C.POINTER(C.c_int32)]
            L.pgs_mvs_select_reference.restype = I
            L.pgs_mvs_depth.argtypes = [P, CamP, CamP, P, P, D, D, P, C.POINTER(I64)]
            L.pgs_mvs_depth.restype = I
            L.pgs_mvs_stage_times.argtypes = [P, CamP, CamP, P, P, D, D, P, P]
            L.pgs_mvs_stage_times.restype = I
            L.pgs_mvs_read.argtypes = [P, C.c_int32, P, I64]
            L.pgs_mvs_read.restype = I
            L.pgs_mvs_fuse.argtypes = [P, CamP, P, P, P, I64, C.POINTER(I64)]
            L.pgs_mvs_fuse.restype = I
            L.pgs_strerror.argtypes = [I]
            L.pgs_strerror.restype = C.c_char_p
            _lib = L
    return _lib


def check(code: int, where: str) -> None:
    if code != PGS_OK:
        raise PgsError(code, where)
