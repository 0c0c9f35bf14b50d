"""Torch-facing wrapper of the C ABI: tensors in, tensors out, the caller's
current CUDA stream.  PyTorch only provides device memory and streams; all
arithmetic runs in libwgeo.so."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


class StaleForwardError(RuntimeError):
    """A backward was asked of a forward whose state the handle no longer holds."""


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev(t: torch.Tensor | None, name: str, shape_last=None):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape_last is not None and (t.dim() < 1 or t.shape[-1] != shape_last):
        raise ValueError(f"{name} must have last dimension {shape_last}")
    return C.c_void_p(t.data_ptr())


def _bbox(bbox) -> C.Array:
    b = np.asarray(bbox, dtype=np.float32).reshape(6)
    return (C.c_float * 6)(*b.tolist())


class Reconstructor:
    """One library handle: workspace for grids up to max_res^3 and clouds of up
    to max_points points, plus the state of its last forward."""

    def __init__(self, max_res: int, max_points: int, device=None, **options):
        self.lib = L.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.opt = L.default_options(**options)
        self.max_res = max_res
        self.max_points = max_points
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.wgeo_create(C.byref(h), max_res, max_points, C.byref(self.opt)),
                    "wgeo_create")
        self.h = h
        self.res = None
        self.n = 0
        # forwards run on this handle so far: the handle keeps only the state
        # of its last forward, so a backward saved against an older forward
        # must be refused (see check_generation)
        self.generation = 0

    @staticmethod
    def footprint(max_res: int, max_points: int, **options) -> int:
        return L.footprint_bytes(max_res, max_points, L.default_options(**options))

    def close(self):
        if self.h:
            self.lib.wgeo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reconstruct(self, points: torch.Tensor, normals: torch.Tensor, bbox, res: int,
                    with_sdf: bool = True, with_normals: bool = True, sdf_out=None, nrm_out=None,
                    stream=None):
        n = int(points.shape[0])
        if normals.shape[0] != n:
            raise ValueError("points and normals differ in length")
        if with_sdf and sdf_out is None:
            sdf_out = torch.empty((res, res, res), device=self.device, dtype=torch.float32)
        if with_normals and nrm_out is None:
            nrm_out = torch.empty((3, res, res, res), device=self.device, dtype=torch.float32)
        rc = self.lib.wgeo_reconstruct(self.h, _dev(points, "points", 3), _dev(normals, "normals", 3),
                                       n, _bbox(bbox), res, _dev(sdf_out, "sdf_out"),
                                       _dev(nrm_out, "nrm_out"), C.c_void_p(_stream(stream)))
        self.generation += 1
        L.check(rc, "wgeo_reconstruct")
        self.res = res
        self.n = n
        return sdf_out, nrm_out

    def check_generation(self, generation: int, what: str = "backward"):
        """Raises StaleForwardError unless the handle's last forward is the one
        numbered `generation` (its state is what a backward differentiates)."""
        if generation != self.generation:
            raise StaleForwardError(
                f"{what}: this Reconstructor has run {self.generation - generation} forward(s) since the "
                f"one being differentiated, and keeps only the last forward's state; give each "
                f"differentiable call its own Reconstructor, or call backward before the next forward")

    def query(self, q: torch.Tensor, with_normals: bool = True, stream=None):
        m = int(q.shape[0])
        sdf_q = torch.empty((m,), device=self.device, dtype=torch.float32)
        nrm_q = torch.empty((m, 3), device=self.device, dtype=torch.float32) if with_normals else None
        rc = self.lib.wgeo_query(self.h, _dev(q, "q", 3), m, _dev(sdf_q, "sdf_q"),
                                 _dev(nrm_q, "nrm_q"), C.c_void_p(_stream(stream)))
        L.check(rc, "wgeo_query")
        return sdf_q, nrm_q

    def query_exact(self, q: torch.Tensor, with_grad: bool = True, stream=None):
        """Exact signed distance to the reconstructed surface at q [m, 3] and
        its gradient (Sec. 2.4 off the grid).  Returns (sdf [m], grad [m, 3] or None)."""
        m = int(q.shape[0])
        sdf_q = torch.empty((m,), device=self.device, dtype=torch.float32)
        grad = torch.empty((m, 3), device=self.device, dtype=torch.float32) if with_grad else None
        rc = self.lib.wgeo_query_exact(self.h, _dev(q, "q", 3), m, _dev(sdf_q, "sdf_q"), _dev(grad, "grad"),
                                       C.c_void_p(_stream(stream)))
        L.check(rc, "wgeo_query_exact")
        return sdf_q, grad

    def backward(self, d_sdf_grid=None, d_nrm_grid=None, q=None, d_sdf_q=None, d_nrm_q=None,
                 want_dq: bool = False, stream=None):
        m = int(q.shape[0]) if q is not None else 0
        d_points = torch.empty((self.n, 3), device=self.device, dtype=torch.float32)
        d_normals = torch.empty((self.n, 3), device=self.device, dtype=torch.float32)
        d_q = torch.empty((m, 3), device=self.device, dtype=torch.float32) if (want_dq and m) else None
        rc = self.lib.wgeo_backward(self.h, _dev(d_sdf_grid, "d_sdf_grid"), _dev(d_nrm_grid, "d_nrm_grid"),
                                    _dev(q, "q"), _dev(d_sdf_q, "d_sdf_q"), _dev(d_nrm_q, "d_nrm_q"), m,
                                    _dev(d_points, "d_points"), _dev(d_normals, "d_normals"),
                                    _dev(d_q, "d_q"), C.c_void_p(_stream(stream)))
        L.check(rc, "wgeo_backward")
        return d_points, d_normals, d_q

    def estimate_normals(self, points: torch.Tensor, bbox, radius: float, eps: float | None = None,
                         with_counts: bool = False, normals_out=None, stream=None):
        """Unoriented D-PCA normals of `points` (Sec. 2.1); eps defaults to
        1e-3 * radius.  Returns (normals [n,3], counts [n] int32 or None)."""
        n = int(points.shape[0])
        if eps is None:
            eps = 1e-3 * radius
        if normals_out is None:
            normals_out = torch.empty((n, 3), device=self.device, dtype=torch.float32)
        counts = torch.empty((n,), device=self.device, dtype=torch.int32) if with_counts else None
        rc = self.lib.wgeo_estimate_normals(self.h, _dev(points, "points", 3), n, _bbox(bbox), float(radius),
                                            float(eps), _dev(normals_out, "normals_out", 3),
                                            C.c_void_p(counts.data_ptr()) if counts is not None else None,
                                            C.c_void_p(_stream(stream)))
        L.check(rc, "wgeo_estimate_normals")
        return normals_out, counts

    def orient_normals(self, points: torch.Tensor, normals: torch.Tensor, bbox, gamma: float = 2.5,
                       n_tol: int = 2, with_stats: bool = False, stream=None):
        """Flips `normals` in place to point out of the sampled surface by
        parity ray casting (Sec. 2.2).  Returns (normals, stats [n,5] int32 or
        None, r_d as a one-element device tensor)."""
        n = int(points.shape[0])
        if normals.shape[0] != n:
            raise ValueError("points and normals differ in length")
        stats = torch.empty((n, 5), device=self.device, dtype=torch.int32) if with_stats else None
        rd = torch.empty((1,), device=self.device, dtype=torch.float32)
        rc = self.lib.wgeo_orient_normals(self.h, _dev(points, "points", 3), n, _bbox(bbox), float(gamma),
                                          int(n_tol), _dev(normals, "normals", 3),
                                          C.c_void_p(stats.data_ptr()) if stats is not None else None,
                                          _dev(rd, "rd"), C.c_void_p(_stream(stream)))
        L.check(rc, "wgeo_orient_normals")
        return normals, stats, rd

    def backward_exact(self, q, d_sdf_q, d_sdf_grid=None, d_nrm_grid=None, want_dq: bool = False,
                       stream=None):
        """Adjoint of exact queries (and optional grid seeds): (d_points,
        d_normals, d_q or None)."""
        m = int(q.shape[0])
        d_points = torch.empty((self.n, 3), device=self.device, dtype=torch.float32)
        d_normals = torch.empty((self.n, 3), device=self.device, dtype=torch.float32)
        d_q = torch.empty((m, 3), device=self.device, dtype=torch.float32) if (want_dq and m) else None
        rc = self.lib.wgeo_backward_exact(self.h, _dev(d_sdf_grid, "d_sdf_grid"), _dev(d_nrm_grid, "d_nrm_grid"),
                                          _dev(q, "q", 3), _dev(d_sdf_q, "d_sdf_q"), m,
                                          _dev(d_points, "d_points"), _dev(d_normals, "d_normals"),
                                          _dev(d_q, "d_q"), C.c_void_p(_stream(stream)))
        L.check(rc, "wgeo_backward_exact")
        return d_points, d_normals, d_q

    def info(self) -> dict:
        inf = L.Info()
        L.check(self.lib.wgeo_get_info(self.h, C.byref(inf)), "wgeo_get_info")
        return {k: getattr(inf, k) for k, _ in L.Info._fields_ if k != "reserved"}

    def field(self, which: str, stream=None) -> torch.Tensor:
        idx = {"b": 0, "chi": 1, "phi": 2, "dphi": 3, "dchi": 4, "lambda": 5, "closest": 6}[which]
        dt = torch.int32 if which == "closest" else torch.float32
        out = torch.empty((self.res, self.res, self.res), device=self.device, dtype=dt)
        r = self.lib.wgeo_get_field(self.h, idx, C.c_void_p(out.data_ptr()), C.c_void_p(_stream(stream)))
        if r < 0:
            L.check(-r, "wgeo_get_field")
        return out

    def stage_times(self, reset: bool = True) -> dict:
        """{stage: (total ms, timed calls)} accumulated since the last reset."""
        ms = np.zeros(len(L.STAGES), dtype=np.float64)
        cnt = np.zeros(len(L.STAGES), dtype=np.int64)
        L.check(self.lib.wgeo_stage_times(self.h, ms.ctypes.data, cnt.ctypes.data, int(reset)),
                "wgeo_stage_times")
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(L.STAGES)}

    def bins(self, stream=None) -> torch.Tensor:
        out = torch.empty((self.n, 3), device=self.device, dtype=torch.int32)
        r = self.lib.wgeo_get_bins(self.h, C.c_void_p(out.data_ptr()), C.c_void_p(_stream(stream)))
        if r < 0:
            L.check(-r, "wgeo_get_bins")
        return out

    def mesh(self):
        T = self.lib.wgeo_get_mesh(self.h, None, None, 0)
        if T < 0:
            L.check(-T, "wgeo_get_mesh")
        verts = np.zeros((T, 3, 3), dtype=np.float32)
        gid = np.zeros((T, 3), dtype=np.int64)
        if T:
            self.lib.wgeo_get_mesh(self.h, verts.ctypes.data, gid.ctypes.data, T)
        return verts, gid


def sh_surface(theta: torch.Tensor, dirs: torch.Tensor, base: float = 0.3, centre=None, stream=None):
    """Points and normals of the SH star body at fixed directions (CUDA)."""
    lib = L.load()
    n = int(dirs.shape[0])
    if centre is None:
        centre = torch.full((3,), 0.5, device=dirs.device, dtype=torch.float32)
    pts = torch.empty((n, 3), device=dirs.device, dtype=torch.float32)
    nrm = torch.empty((n, 3), device=dirs.device, dtype=torch.float32)
    L.check(lib.wgeo_sh_surface(_dev(theta, "theta"), int(theta.numel()), _dev(dirs, "dirs", 3), n,
                                float(base), _dev(centre, "centre"), _dev(pts, "pts"), _dev(nrm, "nrm"),
                                C.c_void_p(_stream(stream))), "wgeo_sh_surface")
    return pts, nrm


def sh_surface_backward(recon: Reconstructor, theta, dirs, d_points, d_normals, base: float = 0.3,
                        stream=None):
    lib = L.load()
    dth = torch.empty_like(theta)
    L.check(lib.wgeo_sh_surface_backward(recon.h, _dev(theta, "theta"), int(theta.numel()),
                                         _dev(dirs, "dirs", 3), int(dirs.shape[0]), float(base),
                                         _dev(d_points, "d_points", 3), _dev(d_normals, "d_normals", 3),
                                         _dev(dth, "d_theta"), C.c_void_p(_stream(stream))),
            "wgeo_sh_surface_backward")
    return dth
