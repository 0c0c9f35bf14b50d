"""Uniform cell-centred grid and point binning (Sec. 2.3, Eq. 16-17 grid; Eq. 25
"central cell").

Grid: ``res`` cells per axis of size h = max_axis(hi - lo) / res over the box
[lo, lo + res*h].  Cell (node) o has centre c_o = lo + (o + 1/2) h.  The
Galerkin unknown a_o of Eq. 16 lives at c_o.

Binning: the central cell of point x is floor((x - lo) / h), clamped into
[0, res - 1], computed with exactly one IEEE subtraction and one IEEE division
in double precision from the float32 inputs.  A point is outside the box when
(x - lo) / h < 0 or > res on some axis (the closed box [lo, lo + res h]).
"""
from __future__ import annotations

import numpy as np

STATUS_POINT_OUTSIDE_BBOX = 1 << 0
STATUS_NONFINITE_INPUT = 1 << 1
STATUS_EMPTY_SURFACE = 1 << 2
STATUS_NOT_CONVERGED = 1 << 3
STATUS_MESH_CAPACITY = 1 << 4


def grid_spacing(bbox, res: int) -> float:
    b = np.asarray(bbox, dtype=np.float32).astype(np.float64)
    return float(max(b[3] - b[0], b[4] - b[1], b[5] - b[2]) / res)


def grid_lo(bbox) -> np.ndarray:
    return np.asarray(bbox, dtype=np.float32)[:3].astype(np.float64)


def node_centres_1d(lo: float, h: float, res: int) -> np.ndarray:
    return lo + (np.arange(res, dtype=np.float64) + 0.5) * h


def node_positions(lo: np.ndarray, h: float, res: int) -> np.ndarray:
    """[res, res, res, 3] array of node centres (x, y, z), indexed [z, y, x]."""
    xs = node_centres_1d(lo[0], h, res)
    ys = node_centres_1d(lo[1], h, res)
    zs = node_centres_1d(lo[2], h, res)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X, Y, Z], axis=-1)


def bin_points(points, bbox, res: int):
    """Central cell (x, y, z) of every point, plus status bits.

    Non-finite points are flagged (and reported through ``finite``); points
    outside the box are flagged and clamped.
    """
    p = np.asarray(points, dtype=np.float32).astype(np.float64)
    lo = grid_lo(bbox)
    h = grid_spacing(bbox, res)
    finite = np.all(np.isfinite(p), axis=1)
    status = 0
    if not finite.all():
        status |= STATUS_NONFINITE_INPUT
    u = (p - lo[None, :]) / h
    with np.errstate(invalid="ignore"):
        fl = np.floor(u)
    fl[~finite] = 0.0
    with np.errstate(invalid="ignore"):
        outside = np.any((u < 0) | (u > res), axis=1) & finite   # closed box [lo, lo + res h]
    if outside.any():
        status |= STATUS_POINT_OUTSIDE_BBOX
    b = np.clip(fl, 0, res - 1).astype(np.int64)
    return b, finite, status
