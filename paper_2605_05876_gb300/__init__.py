"""GB300 (sm_103a) implementation of the differentiable surfel rasteriser of
3D Surface Splatting (arxiv 2605.05876): CUDA kernels behind the C ABI of
include/ss3d.h, with a thin Python binding."""
from . import scenes  # noqa: F401


def build(force: bool = False, verbose: bool = False) -> str:
    from .compile import build as _b
    return _b(force=force, verbose=verbose)
