"""ctypes declarations of libpf.so (include/pf.h).  Argument marshalling only.

The library is built in-tree (paper_2304_07338_b300/libpf.so) by build.py.
Loading fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpf.so")

PF_OK, PF_ERR_INVALID_ARG, PF_ERR_OOM, PF_ERR_CUDA, PF_ERR_TIMEOUT, PF_ERR_UNSUPPORTED, PF_ERR_NUMERIC = range(7)
STATUS_NAMES = ["PF_OK", "PF_ERR_INVALID_ARG", "PF_ERR_OOM", "PF_ERR_CUDA", "PF_ERR_TIMEOUT",
                "PF_ERR_UNSUPPORTED", "PF_ERR_NUMERIC"]


class PfVolume(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dtype", C.c_int),
                ("data_dev", C.c_void_p), ("sigma_scale", C.c_float), ("albedo", C.c_float),
                ("tf_lut_dev", C.c_void_p), ("tf_n", C.c_int), ("majorant", C.c_float),
                ("brick_majorants_dev", C.c_void_p), ("brick", C.c_int),
                ("brick_primary", C.c_int), ("brick_shadow", C.c_int), ("tiled_dev", C.c_void_p)]


class PfLight(C.Structure):
    _fields_ = [("kind", C.c_int), ("v", C.c_float * 3), ("rgb", C.c_float * 3)]


class PfCamera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("at", C.c_float * 3), ("up", C.c_float * 3), ("fovy_deg", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class PfFieldDesc(C.Structure):
    _fields_ = [("in_freqs", C.c_int), ("hidden", C.c_int), ("n_hidden", C.c_int), ("prec", C.c_int),
                ("psi", C.c_float), ("seed", C.c_uint64), ("encoding", C.c_int), ("hash_levels", C.c_int),
                ("hash_features", C.c_int), ("hash_log2_size", C.c_int), ("hash_base_res", C.c_int),
                ("hash_scale", C.c_float)]


class PfTrainDesc(C.Structure):
    _fields_ = [("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("decay", C.c_float), ("decay_start_frac", C.c_float),
                ("decay_every", C.c_int), ("seed", C.c_uint64), ("target", C.c_int), ("knn_k", C.c_int),
                ("knn_stages", C.c_int), ("knn_stage_begin", C.c_float * 8), ("knn_radius", C.c_float * 8)]


class PfCacheInfo(C.Structure):
    _fields_ = [("n_photons", C.c_int64), ("n_records", C.c_int64), ("n_keys", C.c_int64),
                ("n_occupied", C.c_int64), ("res", C.c_int), ("n_lights", C.c_int), ("n_g", C.c_int),
                ("max_bounces", C.c_int), ("tally", C.c_double * 15)]


# name -> (restype, argtypes); the exported symbols of include/pf.h
P, I, I64, U64, F, D = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_float, C.c_double
PP = C.POINTER(C.c_void_p)
SIGNATURES = {
    "pf_create": (I, [PP, I, P]),
    "pf_destroy": (I, [P]),
    "pf_set_stream": (I, [P, P]),
    "pf_last_error": (C.c_char_p, [P]),
    "pf_set_counters": (I, [P, P]),
    "pf_stage_timing": (I, [P, I]),
    "pf_stage_times": (I, [P, C.POINTER(C.c_double), C.POINTER(C.c_int), I]),
    "pf_sync": (I, [P]),
    "pf_volume_majorant": (I, [P, C.POINTER(PfVolume), C.POINTER(C.c_float)]),
    "pf_volume_brick_majorants": (I, [P, C.POINTER(PfVolume), P]),
    "pf_volume_tile": (I, [P, C.POINTER(PfVolume), P]),
    "pf_build_photon_cache": (I, [P, C.POINTER(PfVolume), C.POINTER(PfLight), I, C.POINTER(C.c_float), I, U64, I, I,
                                  U64, I, PP]),
    "pf_cache_info": (I, [P, P, C.POINTER(PfCacheInfo)]),
    "pf_cache_export": (I, [P, P, P, P, P, P, P, P, P, P, P]),
    "pf_cache_free": (I, [P]),
    "pf_sample_queries": (I, [P, P, I64, I, U64, P]),
    "pf_estimate_targets": (I, [P, P, P, I64, F, P, P]),
    "pf_estimate_targets_knn": (I, [P, P, P, I64, I, F, F, P, P, P, P]),
    "pf_field_create": (I, [P, C.POINTER(PfFieldDesc), PP]),
    "pf_field_free": (I, [P]),
    "pf_field_num_params": (I64, [P]),
    "pf_field_get_weights": (I, [P, P, P]),
    "pf_field_set_weights": (I, [P, P, P]),
    "pf_field_calibrate_fp8": (I, [P, P, P, I64]),
    "pf_field_forward": (I, [P, P, P, I64, P]),
    "pf_field_backward": (I, [P, P, P, P, I64, P]),
    "pf_field_encode": (I, [P, P, I64, I, P]),
    "pf_field_loss_gradient": (I, [P, P, P, P, I64, P, P]),
    "pf_field_adam": (I, [P, P, P, F, F, F, F]),
    "pf_train_field": (I, [P, P, C.POINTER(PfTrainDesc), P, P]),
    "pf_render_neural": (I, [P, C.POINTER(PfVolume), C.POINTER(PfLight), I, F, C.POINTER(PfCamera), I, F, U64, P, P]),
    "pf_render_raymarched": (I, [P, C.POINTER(PfVolume), C.POINTER(PfLight), I, F, C.POINTER(PfCamera), I, F, U64, P,
                                 P]),
    "pf_render_pathtraced": (I, [P, C.POINTER(PfVolume), C.POINTER(PfLight), I, F, C.POINTER(PfCamera), I, I, U64, I,
                                 P]),
    "pf_render_pathtraced_noalloc": (I, [C.POINTER(PfVolume), C.POINTER(PfLight), I, F, C.POINTER(PfCamera), I, I,
                                         U64, I, P, P, C.c_char_p, I]),
    "pf_image_rmse": (I, [P, P, P, I64, C.POINTER(C.c_double)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libpf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpf.so not found at %s: build it with `python -m paper_2304_07338_b300.build` "
                           "(the CUDA path has no fallback)" % path)
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status
