"""GB300-native implicit mesh smoothing with adjoint gradients (the inverse mean-curvature-flow
step of "iskra: A System for Inverse Geometry Processing", §7.1, and its linear-solve adjoint,
§5.2).

The compute path is the CUDA library built from csrc/ (see include/iskra_gb300.h); the Python
side only marshals arguments. The native library is loaded on first use and its absence is an
error: there is no CPU fallback.
"""
__all__ = ["meshgen"]
