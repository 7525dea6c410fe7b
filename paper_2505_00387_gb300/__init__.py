"""GB300-native fast azimuthally anisotropic hyperbolic Radon transform.

The operator L (Algorithm 1 of Mokhtari & Gholami, eq. axb2), its exact
adjoint and the sparse FISTA/ISTA solve (eqs. cost1, ISTA, soft) run in
hand-written sm_103a CUDA kernels behind the C ABI of include/aahrt.h
(libaahrt.so).  ``_lib`` binds that ABI under the same names; ``plan``
wraps it for torch tensors; ``autograd`` makes L differentiable.

Importing the package does not load the CUDA library (so the synthetic
input generators work without a GPU); the first plan does, and fails
loudly if it is missing.
"""
__all__ = ["AahrtPlan", "load_library"]


def load_library():
    from . import _lib
    return _lib.load()


def __getattr__(name):
    if name == "AahrtPlan":
        from .plan import AahrtPlan
        return AahrtPlan
    raise AttributeError(name)
