"""ctypes loader of libspf.so (the C ABI declared in include/spf.h).

Argument marshalling only. If the shared library is missing this module
raises at import time: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspf.so")

SPF_OK = 0
SPF_ERR_ARG = -1
SPF_ERR_OOM = -2
SPF_ERR_CUDA = -3
SPF_ERR_TIMEOUT = -4
SPF_ERR_UNSUPPORTED = -5
SPF_FP32, SPF_BF16, SPF_FP8 = 0, 1, 2
SPF_IMAGES_F32, SPF_IMAGES_U16 = 0, 1
SPF_UPLOAD_COPY, SPF_UPLOAD_SM = 0, 1
SPF_PHASE_ER, SPF_PHASE_HIO = 0, 1

_CODES = {SPF_ERR_ARG: "SPF_ERR_ARG", SPF_ERR_OOM: "SPF_ERR_OOM", SPF_ERR_CUDA: "SPF_ERR_CUDA",
          SPF_ERR_TIMEOUT: "SPF_ERR_TIMEOUT", SPF_ERR_UNSUPPORTED: "SPF_ERR_UNSUPPORTED"}


class SpfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


P = C.c_void_p
I = C.c_int
I64 = C.c_int64
F = C.c_float
D = C.c_double

class MtipConfig(C.Structure):
    """spf_mtip_config (include/spf.h)."""
    _fields_ = [("N", C.c_int), ("qmax", C.c_double), ("eps", C.c_double), ("P2", C.c_int),
                ("max_images", C.c_int), ("n_orient", C.c_int), ("orient_chunk", C.c_int),
                ("img_chunk", C.c_int), ("precision", C.c_int), ("topk", C.c_int), ("cache_points", C.c_int),
                ("point_budget_bytes", C.c_int64), ("host_image_type", C.c_int), ("device", C.c_int),
                ("keep_slices", C.c_int)]


# name: (restype, argtypes)
PROTOTYPES = {
    "spf_last_error_string": (C.c_char_p, []),
    "spf_version": (I, []),
    "spf_plan_create": (I, [C.POINTER(P), I, D, D, I64, I]),
    "spf_plan_destroy": (I, [P]),
    "spf_plan_status": (I, [P]),
    "spf_plan_sizes": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
    "spf_slice_model": (I, [P, P, P, I, P, I, P, P]),
    "spf_slice_adjoint": (I, [P, P, P, I, P, I, P, I, P]),
    "spf_nufft_type2": (I, [P, P, P, I64, P, P]),
    "spf_nufft_type1": (I, [P, P, P, I64, P, I, P]),
    "spf_merge_images": (I, [P, P, P, I, P, I, P, I, P, F, P, P, I, P]),
    "spf_points_create": (I, [C.POINTER(P), P, P, I, P, I, I, P]),
    "spf_points_destroy": (I, [P]),
    "spf_slice_points": (I, [P, P, P, P, P]),
    "spf_merge_points": (I, [P, P, P, P, I, I, P, F, P, P, I, P]),
    "spf_merge_begin": (I, [P, P]),
    "spf_merge_points_add": (I, [P, P, P, P, I, I, P, F, I, I, P]),
    "spf_merge_images_add": (I, [P, P, P, I, P, I, P, I, P, F, I, I, P]),
    "spf_merge_finish": (I, [P, P, P, I, P]),
    "spf_cg_begin": (I, [P, P, D, P, P, P, P, P]),
    "spf_cg_merge_step": (I, [P, P, D, P, P, P]),
    "spf_toeplitz_apply": (I, [P, P, D, P, P, P]),
    "spf_slice_loss_grad": (I, [P, P, P, P, I, P, I, P, F, P, D, I, P, P, P, P]),
    "spf_slice_normal_apply": (I, [P, P, P, I, P, I, P, D, I, P, P, P]),
    "spf_gradient_step": (I, [P, P, P, P, I, P, I, P, F, P, D, I, P, P, P, P, P]),
    "spf_cg_objective": (I, [P, P, P, P, P, P, P, P]),
    "spf_weighted_sumsq": (I, [P, P, I, I, P, F, P, I, P]),
    "spf_lcurve_corner": (I, [P, P, P, I, C.POINTER(I), P]),
    "spf_matcher_create": (I, [C.POINTER(P), I, I, I, I, I, I]),
    "spf_matcher_destroy": (I, [P]),
    "spf_matcher_status": (I, [P]),
    "spf_matcher_set_images": (I, [P, P, I, F, P]),
    "spf_matcher_set_images_u16": (I, [P, P, I, F, P]),
    "spf_matcher_set_mask": (I, [P, P, P]),
    "spf_matcher_add_slices": (I, [P, P, I, I, P]),
    "spf_matcher_set_schedule": (I, [P, I]),
    "spf_matcher_set_rerank": (I, [P, I]),
    "spf_matcher_results": (I, [P, P, P, P, P, P, P]),
    "spf_match_orientations": (I, [P, P, I, F, P, I, P, P, P, P]),
    "spf_match_orientations_static": (I, [P, I, F, P, I, I, P, P, P, P]),
    "spf_counts_to_f32": (I, [P, I64, P, P]),
    "spf_morton_order": (I, [P, I, P]),
    "spf_phaser_create": (I, [C.POINTER(P), I, I]),
    "spf_phaser_destroy": (I, [P]),
    "spf_phaser_set_amplitudes": (I, [P, P, P]),
    "spf_phaser_amplitudes_from_model": (I, [P, P, P]),
    "spf_phaser_set_state": (I, [P, P, P, P]),
    "spf_phaser_iterate": (I, [P, I, I, F, I, P, P]),
    "spf_phaser_shrinkwrap": (I, [P, F, F, P]),
    "spf_phaser_get": (I, [P, P, P, P, P]),
    "spf_mtip_create": (I, [C.POINTER(P), C.POINTER(MtipConfig)]),
    "spf_mtip_destroy": (I, [P]),
    "spf_mtip_info": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(I), C.POINTER(I)]),
    "spf_mtip_plan": (P, [P]),
    "spf_mtip_matcher": (P, [P]),
    "spf_mtip_status": (I, [P]),
    "spf_mtip_set_orientations": (I, [P, P, P, P]),
    "spf_mtip_set_mask": (I, [P, P, P]),
    "spf_mtip_match": (I, [P, P, P, I, I, F, P, P, P, P, P, P]),
    "spf_mtip_merge": (I, [P, P, I, I, F, P, P, P, P]),
    "spf_mtip_solve": (I, [P, P, P, P, D, I64, I, P, C.POINTER(D), P, P]),
    "spf_mtip_iteration": (I, [P, P, P, I, I, F, I, D, P, P, C.POINTER(D), P]),
    "spf_mtip_iteration_host": (I, [P, P, P, I, I, F, I, D, P, P, C.POINTER(D), P]),
    "spf_mtip_set_upload": (I, [P, I]),
    "spf_mtip_upload_host": (I, [P, P, P, I, I, C.POINTER(P), C.POINTER(P), P]),
    "spf_mtip_release_upload": (I, [P, P]),
    "spf_mtip_last_upload_ms": (I, [P, C.POINTER(F)]),
    "spf_profile_enable": (I, [I]),
    "spf_profile_select": (I, [C.c_char_p]),
    "spf_profile_read": (I, [I, C.c_char_p, I, C.POINTER(C.c_longlong), C.POINTER(D)]),
    "spf_profile_bytes": (I, [I, C.POINTER(D)]),
    "spf_launch_count": (C.c_longlong, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2109_05339_gb300.build` "
            "(nvcc for sm_103a). There is no fallback implementation.")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def check(code):
    if code != SPF_OK:
        msg = lib.spf_last_error_string()
        raise SpfError(code, msg.decode() if msg else "")
    return code


def profile_enable(on=True):
    lib.spf_profile_enable(1 if on else 0)


def profile_select(names=None):
    """Trace only the named kernels (None: all)."""
    lib.spf_profile_select(",".join(names).encode() if names else None)


def profile_read():
    """{kernel name: (launches, total device ms)} since the last profile_enable()."""
    out = {}
    i = 0
    buf = C.create_string_buffer(128)
    n, ms = C.c_longlong(), C.c_double()
    while lib.spf_profile_read(i, buf, 128, C.byref(n), C.byref(ms)) == SPF_OK:
        out[buf.value.decode()] = (n.value, ms.value)
        i += 1
    return out


def profile_bytes():
    """{kernel name: algorithmic bytes of its traced launches} since the last
    profile_enable() (0 for kernels that state none)."""
    out = {}
    i = 0
    buf = C.create_string_buffer(128)
    n, ms, b = C.c_longlong(), C.c_double(), C.c_double()
    while lib.spf_profile_read(i, buf, 128, C.byref(n), C.byref(ms)) == SPF_OK:
        if lib.spf_profile_bytes(i, C.byref(b)) == SPF_OK:
            out[buf.value.decode()] = b.value
        i += 1
    return out


def launch_count():
    return int(lib.spf_launch_count())
