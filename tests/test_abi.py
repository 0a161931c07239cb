"""The C-ABI library loads on a machine without a GPU, exports every function
that include/*.h declares, and rejects bad arguments before touching CUDA."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(spf_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2109_05339_gb300 import build
    build.build()
    from paper_2109_05339_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = names - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    assert names == set(lib.PROTOTYPES), "binding prototypes differ from the header"


def test_argument_errors_without_gpu(lib):
    L = lib.lib
    h = C.c_void_p()
    assert L.spf_plan_create(C.byref(h), 16, 1.0, 1e-6, 0, 0) == lib.SPF_ERR_ARG   # even N
    assert b"odd" in L.spf_last_error_string()
    assert L.spf_plan_create(C.byref(h), 17, 1.0, 1e-9, 0, 0) == lib.SPF_ERR_ARG   # eps
    assert L.spf_plan_create(C.byref(h), 17, -1.0, 1e-6, 0, 0) == lib.SPF_ERR_ARG  # qmax
    assert L.spf_plan_create(None, 17, 1.0, 1e-6, 0, 0) == lib.SPF_ERR_ARG
    assert L.spf_slice_model(None, None, None, 1, None, 1, None, None) == lib.SPF_ERR_ARG
    assert L.spf_cg_merge_step(None, None, 0.0, None, None, None) == lib.SPF_ERR_ARG
    m = C.c_void_p()
    assert L.spf_matcher_create(C.byref(m), 10, 10, 16, 7, 8, 0) == lib.SPF_ERR_ARG  # precision
    assert L.spf_matcher_create(C.byref(m), 10, 10, 16, 0, 9, 0) == lib.SPF_ERR_ARG  # topk
    assert L.spf_matcher_add_slices(None, None, 1, 0, None) == lib.SPF_ERR_ARG
    assert L.spf_counts_to_f32(None, 8, None, None) == lib.SPF_ERR_ARG      # NULL buffers
    assert L.spf_counts_to_f32(None, -1, None, None) == lib.SPF_ERR_ARG     # negative size
    # odd address; with n = 0 nothing would be read even if the check were lost
    # an odd (misaligned) address of a real host buffer: rejected before any use
    buf = (C.c_uint8 * 64)()
    odd = C.c_void_p(C.addressof(buf) + 1)
    assert L.spf_counts_to_f32(odd, 0, C.c_void_p(C.addressof(buf) + 16), None) == lib.SPF_ERR_ARG
    assert L.spf_version() == 1
    # destroying NULL handles is a no-op
    assert L.spf_plan_destroy(None) == 0 and L.spf_matcher_destroy(None) == 0


def test_driver_configuration_errors_without_gpu(lib):
    """spf_mtip_create checks its configuration before any CUDA call: the
    point-set mode (-1, 0, 1 or 2) and an orientation chunk whose points reach
    2^31 (the paper's 1.2e6 orientations of 128 x 128 pixels at once)."""
    L = lib.lib

    def cfg(**kw):
        base = dict(N=17, qmax=1.0, eps=1e-6, P2=256, max_images=10, n_orient=100, orient_chunk=0, img_chunk=0,
                    precision=1, topk=8, cache_points=-1, point_budget_bytes=0, host_image_type=-1, device=0,
                    keep_slices=-1)
        base.update(kw)
        return lib.MtipConfig(**base)

    h = C.c_void_p()
    assert L.spf_mtip_create(C.byref(h), C.byref(cfg(cache_points=3))) == lib.SPF_ERR_ARG
    assert b"cache_points" in L.spf_last_error_string()
    assert L.spf_mtip_create(C.byref(h), C.byref(cfg(cache_points=-2))) == lib.SPF_ERR_ARG
    big = cfg(P2=16384, n_orient=1_200_000)
    assert L.spf_mtip_create(C.byref(h), C.byref(big)) == lib.SPF_ERR_ARG
    assert b"2^31" in L.spf_last_error_string()
    assert L.spf_mtip_create(C.byref(h), C.byref(cfg(orient_chunk=-1))) == lib.SPF_ERR_ARG
    assert not h.value


def test_binding_raises_typed_errors(lib):
    with pytest.raises(lib.SpfError) as e:
        lib.check(lib.SPF_ERR_ARG)
    assert e.value.code == lib.SPF_ERR_ARG
