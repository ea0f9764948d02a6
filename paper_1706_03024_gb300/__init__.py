"""GB300 (sm_103a) light tracer for highly scattering fluorescent participating media.

Method: Abdellah et al., arXiv 1706.03024. The compute path is libfluoro.so (CUDA kernels behind
the C ABI in include/fluoro.h); `native` binds it with ctypes and `scene` marshals scene
descriptions onto it. Importing the package does not load the library; the first call does, and
raises if it is missing.
"""
from . import build  # noqa: F401

__all__ = ["build", "native", "scene", "shard", "units"]


def __getattr__(name):
    if name in ("native", "scene", "shard", "units"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
