"""GB300-native implicit mesh smoothing with adjoint gradients (the inverse mean-curvature-flow
step of "iskra: A System for Inverse Geometry Processing", §7.1, and its linear-solve adjoint,
§5.2).

The compute path is the CUDA library built from csrc/ (declared in include/iskra_gb300.h); the
Python side only marshals arguments. The native library is loaded on first use and its absence
is an error: there is no CPU fallback.
"""
from importlib import import_module

__all__ = ["meshgen", "api", "Mesh", "Context", "smooth", "make_opts", "build_native"]


def build_native(force: bool = False) -> str:
    from . import build as _b
    return _b.build(force=force)


def __getattr__(name):
    if name in ("Mesh", "Context", "smooth", "make_opts", "SmoothSolve", "default_context"):
        return getattr(import_module(".api", __name__), name)
    if name in ("meshgen", "api", "build"):
        return import_module("." + name, __name__)
    raise AttributeError(name)
