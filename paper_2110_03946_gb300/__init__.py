"""GB300-native multilevel ORAS solver for homogeneous diffusion inpainting.

Kaemper & Weickert, "Domain decomposition algorithms for real-time homogeneous
diffusion inpainting in 4K" (arXiv 2110.03946).  The solver is a CUDA library
for sm_103a with a C ABI (include/dd_inpaint.h); ``binding`` is its ctypes
binding and ``inpaint`` a torch-tensor convenience layer.  There is no CPU
fallback: without the built library the calls raise.
"""
from . import binding  # noqa: F401

__all__ = ["binding", "build_library", "Inpainter", "inpaint"]


def build_library(force: bool = False) -> str:
    from .build import build
    return build(force=force)


def __getattr__(name):
    if name in ("Inpainter", "inpaint", "make_params"):
        from . import inpaint as _m
        return getattr(_m, name)
    raise AttributeError(name)
