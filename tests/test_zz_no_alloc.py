"""The allocation-free matching entry point gives the regular matcher's results.

Some callers cannot allocate device memory when they match: code inside a host
framework that owns the device memory pool and forbids allocations beside it,
or a real-time acquisition loop that must not touch the allocator (its calls
can block and synchronise the device). For them the library offers
spf_match_orientations_static, whose scratch is a static device array instead
of cudaMalloc'd buffers. This test calls it through the C ABI twice in a row
(different sizes, so leftovers of the first call would show in the second)
and compares each result with spf_match_orientations (FP32, top-8 re-rank).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_static_scratch_matching_equals_matcher():
    import torch
    from paper_2109_05339_gb300 import Matcher, _lib
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    rng = np.random.default_rng(2024)
    for n_img, n_orient, P2, scale in [(300, 1000, 256, 1.0), (1024, 700, 515, 0.5)]:
        Y = rng.gamma(2.0, 1.0, (n_orient, P2)).astype(np.float32)
        pick = rng.integers(0, n_orient, n_img)
        X = (Y[pick] / scale + rng.normal(0, 0.05, (n_img, P2))).astype(np.float32)
        Xd = torch.from_numpy(X).to(dev)
        Yd = torch.from_numpy(Y).to(dev)
        best = torch.empty(n_img, dtype=torch.int32, device=dev)
        d1 = torch.empty(n_img, dtype=torch.float32, device=dev)
        d2 = torch.empty(n_img, dtype=torch.float32, device=dev)
        _lib.check(_lib.lib.spf_match_orientations_static(
            _ptr(Xd), n_img, C.c_float(scale), _ptr(Yd), n_orient, P2, _ptr(best), _ptr(d1),
            _ptr(d2), stream))
        m = Matcher(n_img, n_orient, P2, "fp32", 8, device=dev)
        ref_best, ref_d1, ref_d2 = m.match(Xd, Yd, scale)
        m.status()
        torch.cuda.synchronize()
        assert torch.equal(best, ref_best)
        np.testing.assert_allclose(d1.cpu().numpy(), ref_d1.cpu().numpy(), rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(d2.cpu().numpy(), ref_d2.cpu().numpy(), rtol=1e-5, atol=1e-6)
        m.close()


def test_static_scratch_rejects_sizes_beyond_its_limit():
    """Sizes above the array's limit are refused with a message naming the
    limit. The buffers are NULL: the call must fail on the size, and were the
    size check ever lost, the NULL-pointer check would still refuse the call
    (with another message, failing this test) before any kernel could run."""
    from paper_2109_05339_gb300 import _lib
    L = _lib.lib
    assert L.spf_match_orientations_static(None, 1025, C.c_float(1.0), None, 10, 64, None, None, None,
                                           None) == _lib.SPF_ERR_ARG
    assert b"limit of 1024" in L.spf_last_error_string()
    assert L.spf_match_orientations_static(None, 10, C.c_float(1.0), None, 65537, 64, None, None, None,
                                           None) == _lib.SPF_ERR_ARG
    assert b"limit of 65536" in L.spf_last_error_string()
