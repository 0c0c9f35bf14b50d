"""Trilinear interpolation on the node lattice and the iso-value (Sec. 2.4, Eq. 27).

chi_h is sampled at the cell centres c_o.  Between centres it is interpolated
trilinearly; a position is first clamped into the node hull
[lo + h/2, lo + (res - 1/2) h] per axis (no extrapolation), and the clamped
axes carry zero derivative.

Iso-value reading: c is the plain mean of the interpolated chi at the input
samples (the Kazhdan 2006 choice the paper cites for Eq. 27).
"""
from __future__ import annotations

import numpy as np


def trilinear(x, lo, h, res):
    """Corner nodes [n,8,3] (x,y,z), weights [n,8], d weight/dx [n,8,3]."""
    p = np.asarray(x, dtype=np.float64)
    u = (p - lo[None, :]) / h - 0.5
    clamped = (u < 0.0) | (u > res - 1)
    u = np.clip(u, 0.0, res - 1)
    i0 = np.minimum(np.floor(u), res - 2).astype(np.int64)
    t = u - i0
    corners = np.zeros((p.shape[0], 8, 3), dtype=np.int64)
    w = np.ones((p.shape[0], 8))
    dw = np.ones((p.shape[0], 8, 3))
    for c in range(8):
        bits = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        corners[:, c, :] = i0 + bits[None, :]
        for ax in range(3):
            f = t[:, ax] if bits[ax] else 1.0 - t[:, ax]
            df = np.where(clamped[:, ax], 0.0, (1.0 if bits[ax] else -1.0) / h)
            w[:, c] *= f
            for ax2 in range(3):
                dw[:, c, ax2] *= df if ax2 == ax else f
    return corners, w, dw


def gather(grid, corners):
    """grid[z,y,x] at corner (x,y,z) indices -> [n, 8] (or [n, 8, C])."""
    return grid[corners[..., 2], corners[..., 1], corners[..., 0]]


def interpolate(grid, x, lo, h, res):
    corners, w, _ = trilinear(x, lo, h, res)
    vals = gather(grid, corners)
    if vals.ndim == 3:
        return np.einsum("nc,nck->nk", w, vals)
    return np.sum(w * vals, axis=1)


def isovalue(chi, points, finite, lo, h, res):
    p = np.asarray(points, dtype=np.float64)[finite]
    if p.shape[0] == 0:
        return 0.0
    return float(np.mean(interpolate(chi, p, lo, h, res)))
