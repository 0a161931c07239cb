"""GB300 (sm_103a) implementation of the data-parallel path of Cartesian-NUFFT
M-TIP reconstruction (arXiv 2109.05339, Sec. II): type-2 NUFFT slicing,
tensor-core orientation matching with FP32 re-ranking, and type-1 NUFFT
merging inside a Toeplitz conjugate-gradient solve.

The compute runs in libspf.so (C ABI in include/spf.h); this package only
marshals PyTorch tensors to it. Accessing any compute entry point loads the
library and raises if it is absent (there is no fallback). The ``build``
submodule compiles it and does not need it.
"""
import importlib

_EXPORTS = {
    "Plan": "api", "PointSet": "api", "Matcher": "api", "SliceModel": "api", "slice_model": "api",
    "SpfError": "api", "PRECISIONS": "api", "counts_to_f32": "api", "MTIP": "mtip", "Phaser": "phasing",
}


def __getattr__(name):
    if name in _EXPORTS:
        mod = importlib.import_module(f".{_EXPORTS[name]}", __name__)
        return getattr(mod, name)
    raise AttributeError(name)


__all__ = list(_EXPORTS)
