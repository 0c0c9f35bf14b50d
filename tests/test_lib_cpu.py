"""CPU-only checks of the C ABI library: it builds, loads, exports every symbol
the header declares, and its host-side logic (options, footprint, error text,
the marching-cubes table it derives) behaves.  No GPU compute is called."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_20964_gb300 import build as B
    B.build_library()
    from paper_2609_20964_gb300 import _lib
    return _lib.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "wgeo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wgeo_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 15
    from paper_2609_20964_gb300 import _lib
    for nm in names:
        assert hasattr(lib, nm), f"{nm} declared in include/wgeo.h but not exported"
        assert nm in _lib.SIGNATURES, f"{nm} has no binding"


def test_default_options_and_footprint(lib):
    from paper_2609_20964_gb300 import _lib
    o = _lib.default_options()
    assert o.tol_rel == 1e-6 and o.precision == _lib.PREC_MIXED and o.keep_for_backward == 1
    f64 = _lib.footprint_bytes(64, 10_000, o)
    f128 = _lib.footprint_bytes(128, 10_000, o)
    f256 = _lib.footprint_bytes(256, 200_000, o)
    assert 0 < f64 < f128 < f256
    # dominated by the res^3 fields, 72 bytes per cell when gradients are kept
    # (b, chi32, float-float chi pair, r, e, phi, closest triangle, dphi (4),
    # dchi (8), float-float lambda pair, lambda32), plus triangles, pucks and points
    assert 72 * 256 ** 3 < f256 < 110 * 256 ** 3
    o2 = _lib.default_options(keep_for_backward=0)
    assert _lib.footprint_bytes(256, 200_000, o2) < f256
    # invalid bounds -> 0
    assert _lib.footprint_bytes(3, 10, o) == 0
    assert _lib.footprint_bytes(100, 10, o) == 0          # coarsens to 25^3 > 16^3
    assert _lib.footprint_bytes(192, 10, o) > 0           # 192 -> 3


def test_error_strings(lib):
    assert lib.wgeo_error_string(0) == b"ok"
    assert b"invalid" in lib.wgeo_error_string(1)
    assert lib.wgeo_status_string(0) == b"ok"
    assert b"capacity" in lib.wgeo_status_string(1 << 4)


def test_null_and_bad_args_rejected_on_host(lib):
    h = C.c_void_p()
    assert lib.wgeo_create(None, 64, 10, None) == 1
    assert lib.wgeo_create(C.byref(h), 3, 10, None) == 1
    assert lib.wgeo_reconstruct(None, None, None, 0, None, 64, None, None, None) == 1
    assert lib.wgeo_query(None, None, 0, None, None, None) == 1
    assert lib.wgeo_backward(None, None, None, None, None, None, 0, None, None, None, None) == 1
    assert lib.wgeo_get_info(None, None) == 1
    # the entry points of the NEXT rows reject a null handle before any device call
    assert lib.wgeo_query_exact(None, None, 0, None, None, None) == 1
    assert lib.wgeo_backward_exact(None, None, None, None, None, 0, None, None, None, None) == 1
    assert lib.wgeo_estimate_normals(None, None, 0, None, 0.1, 1e-4, None, None, None) == 1
    assert lib.wgeo_orient_normals(None, None, 0, None, 2.5, 2, None, None, None, None) == 1


def test_library_mc_table_equals_oracle_golden(lib):
    # the library derives its table with its own code; it must agree with the
    # table the oracle derives (stored under tests/golden by the oracle script)
    from paper_2609_20964_gb300 import _lib
    counts, tris = _lib.mc_table()
    with open(os.path.join(ROOT, "tests", "golden", "mc_table.txt")) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    assert len(lines) == 256
    for c in range(256):
        want = [int(v) for v in lines[c].split()] if lines[c] else []
        got = tris[c, :counts[c]].reshape(-1).tolist()
        assert got == want, f"case {c}"
        assert np.all(tris[c, counts[c]:] == -1)


def test_python_layer_names():
    # the autograd entry and the serving loop are importable without a GPU
    torch = pytest.importorskip("torch")
    import paper_2609_20964_gb300 as W
    assert issubclass(W.WgeoFunction, torch.autograd.Function)
    assert W.WgeoFunction is W.WgeoQueryFunction
    assert callable(W.Server) and hasattr(W.Server, "submit")
