"""GB300-native (sm_103a) differentiable SDF reconstruction from oriented point
clouds: 27-cell normal splat, divergence, Poisson solve, iso-value, marching
cubes, exact signed distance, stencil normals and their adjoints, all in the
CUDA library ``_build/libwgeo.so`` behind the C ABI of ``include/wgeo.h``.

Importing this package does not load the library; the first Reconstructor
does, and raises if it has not been built.
"""
from ._lib import (  # noqa: F401
    PREC_FP32,
    PREC_FP64,
    PREC_MIXED,
    STATUS_EMPTY_SURFACE,
    STATUS_MESH_CAPACITY,
    STATUS_NONFINITE_INPUT,
    STATUS_NOT_CONVERGED,
    STATUS_POINT_OUTSIDE_BBOX,
    WgeoError,
    load,
    mc_table,
)


def __getattr__(name):
    # torch-dependent parts load lazily so that the CPU-only symbol checks need no torch import
    if name in ("Reconstructor", "sh_surface", "sh_surface_backward", "StaleForwardError"):
        from . import api
        return getattr(api, name)
    if name in ("sdf_query", "sdf_query_exact", "sdf_grid", "sh_points", "WgeoFunction", "WgeoQueryFunction",
                "WgeoExactQueryFunction", "WgeoGridFunction", "SHSurfaceFunction"):
        from . import autograd
        return getattr(autograd, name)
    if name in ("Server", "Request"):
        from . import serving
        return getattr(serving, name)
    raise AttributeError(name)
