"""GB300-native edge-based grid metrics (arXiv 2502.00778).

Lumped directed-area vectors at edges, median-dual volumes and boundary
dual-face normals of triangular/tetrahedral grids, computed straight from
element geometry, plus their adjoint -- hand-written CUDA for sm_103a behind
the C ABI in include/edgemetrics.h.
"""
from ._lib import EMError, PATH, PREC, load  # noqa: F401

__all__ = ["EMError", "PATH", "PREC", "load", "api"]


def __getattr__(name):
    # import the torch-based binding lazily so the C-ABI symbol checks run
    # without importing torch
    if name == "api":
        import importlib
        return importlib.import_module(__name__ + ".api")
    raise AttributeError(name)
