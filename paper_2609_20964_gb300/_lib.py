"""ctypes binding of the C ABI in include/wgeo.h — argument marshalling only.

Every compute step runs in the CUDA library ``_build/libwgeo.so``.  Loading
fails loudly if the library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwgeo.so")

WGEO_OK = 0
WGEO_ERR_INVALID_ARG = 1
WGEO_ERR_OOM = 2
WGEO_ERR_CUDA = 3
WGEO_ERR_NO_FORWARD = 4
WGEO_ERR_NOT_BUILT_FOR_DEVICE = 5

STATUS_POINT_OUTSIDE_BBOX = 1 << 0
STATUS_NONFINITE_INPUT = 1 << 1
STATUS_EMPTY_SURFACE = 1 << 2
STATUS_NOT_CONVERGED = 1 << 3
STATUS_MESH_CAPACITY = 1 << 4

STAGES = ("splat", "solve", "iso", "mc", "sdf", "normals", "query", "bwd_seed",
          "bwd_surface", "bwd_solve", "bwd_splat", "sdf_tie", "point_pca", "orient", "query_exact")

PREC_MIXED = 0
PREC_FP32 = 1
PREC_FP64 = 2

# every function the header declares, with (restype, argtypes)
_vp = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64
_f32 = C.c_float


class Options(C.Structure):
    _fields_ = [("tol_rel", C.c_double), ("max_vcycles", _i32), ("max_refine", _i32),
                ("vcycles_per_refine", _i32), ("precision", _i32), ("warm_start", _i32),
                ("keep_for_backward", _i32), ("mesh_capacity", _i64), ("use_graphs", _i32),
                ("stage_timing", _i32), ("galerkin", _i32), ("spectral", _i32), ("reserved", _i32 * 3),
                ("tol_rel_adjoint", C.c_double)]


class Info(C.Structure):
    _fields_ = [("status", C.c_uint32), ("res", _i32), ("solver_steps", _i32),
                ("backward_steps", _i32), ("residual_rel", C.c_double),
                ("backward_residual_rel", C.c_double), ("isovalue", C.c_double),
                ("n_triangles", _i64), ("n_points_used", _i64), ("h", C.c_double),
                ("sdf_node_visits", _i64), ("sdf_leaf_visits", _i64), ("sdf_tri_tests", _i64),
                ("backward_dc", C.c_double), ("sdf_tie_nodes", _i64), ("reserved", _i64 * 1)]


SIGNATURES = {
    "wgeo_default_options": (C.c_int, [C.POINTER(Options)]),
    "wgeo_footprint_bytes": (C.c_size_t, [_i32, _i64, C.POINTER(Options)]),
    "wgeo_create": (C.c_int, [C.POINTER(_vp), _i32, _i64, C.POINTER(Options)]),
    "wgeo_destroy": (C.c_int, [_vp]),
    "wgeo_reconstruct": (C.c_int, [_vp, _vp, _vp, _i64, C.POINTER(_f32), _i32, _vp, _vp, _vp]),
    "wgeo_query": (C.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "wgeo_query_exact": (C.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
    "wgeo_backward_exact": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "wgeo_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "wgeo_estimate_normals": (C.c_int, [_vp, _vp, _i64, C.POINTER(_f32), _f32, _f32, _vp, _vp, _vp]),
    "wgeo_orient_normals": (C.c_int, [_vp, _vp, _i64, C.POINTER(_f32), _f32, _i32, _vp, _vp, _vp, _vp]),
    "wgeo_get_info": (C.c_int, [_vp, C.POINTER(Info)]),
    "wgeo_get_field": (_i64, [_vp, _i32, _vp, _vp]),
    "wgeo_get_mesh": (_i64, [_vp, _vp, _vp, _i64]),
    "wgeo_get_bins": (_i64, [_vp, _vp, _vp]),
    "wgeo_mc_table": (C.c_int, [_vp, _vp]),
    "wgeo_sh_surface": (C.c_int, [_vp, _i32, _vp, _i64, _f32, _vp, _vp, _vp, _vp]),
    "wgeo_sh_surface_backward": (C.c_int, [_vp, _vp, _i32, _vp, _i64, _f32, _vp, _vp, _vp, _vp]),
    "wgeo_sh_surface_backward_noalloc": (C.c_int, [_vp, _i32, _vp, _i64, _f32, _vp, _vp, _vp, _vp]),
    "wgeo_stage_times": (C.c_int, [_vp, _vp, _vp, _i32]),
    "wgeo_kernel_launches": (_i64, []),
    "wgeo_error_string": (C.c_char_p, [C.c_int]),
    "wgeo_status_string": (C.c_char_p, [C.c_uint32]),
}

_LIB = None


def load(path: str = LIB_PATH):
    """Load libwgeo.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class WgeoError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        super().__init__(f"{where}: {lib.wgeo_error_string(code).decode()} (code {code})")
        self.code = code


def check(code: int, where: str):
    if code != WGEO_OK:
        raise WgeoError(code, where)


def default_options(**kw) -> Options:
    o = Options()
    check(load().wgeo_default_options(C.byref(o)), "wgeo_default_options")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def footprint_bytes(max_res: int, max_points: int, opt: Options | None = None) -> int:
    return int(load().wgeo_footprint_bytes(max_res, max_points, C.byref(opt) if opt else None))


def mc_table():
    import numpy as np
    counts = np.zeros(256, dtype=np.int32)
    tris = np.zeros((256, 5, 3), dtype=np.int32)
    check(load().wgeo_mc_table(counts.ctypes.data, tris.ctypes.data), "wgeo_mc_table")
    return counts, tris
