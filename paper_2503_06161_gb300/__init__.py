"""GB300 (sm_103a) FE-4DGS differentiable rasterization pass.

The CUDA library is loaded lazily, on first use of a rendering function, so
that ``paper_2503_06161_gb300.synth`` and ``.build`` import without a GPU.
"""
__all__ = ["build", "synth", "raster"]


def __getattr__(name):
    if name == "raster":
        from . import raster
        return raster
    raise AttributeError(name)
