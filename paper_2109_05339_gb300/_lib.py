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
    "spf_cg_begin": (I, [P, P, D, P, P, P, P, P]),
    "spf_cg_merge_step": (I, [P, P, D, P, P, P]),
    "spf_toeplitz_apply": (I, [P, P, D, P, P, P]),
    "spf_cg_objective": (I, [P, P, P, P, P, P, P, P]),
    "spf_weighted_sumsq": (I, [P, P, I, I, P, F, P, I, P]),
    "spf_matcher_create": (I, [C.POINTER(P), I, I, I, I, I, I]),
    "spf_matcher_destroy": (I, [P]),
    "spf_matcher_status": (I, [P]),
    "spf_matcher_set_images": (I, [P, P, I, F, P]),
    "spf_matcher_set_mask": (I, [P, P, P]),
    "spf_matcher_add_slices": (I, [P, P, I, I, P]),
    "spf_matcher_results": (I, [P, P, P, P, P, P, P]),
    "spf_match_orientations": (I, [P, P, I, F, P, I, P, P, P, P]),
    "spf_match_orientations_static": (I, [P, I, F, P, I, I, P, P, P, P]),
    "spf_counts_to_f32": (I, [P, I64, P, P]),
    "spf_profile_enable": (I, [I]),
    "spf_profile_select": (I, [C.c_char_p]),
    "spf_profile_read": (I, [I, C.c_char_p, I, C.POINTER(C.c_longlong), C.POINTER(D)]),
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


def launch_count():
    return int(lib.spf_launch_count())
