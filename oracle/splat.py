"""27-cell normal splat (Sec. 2.3, Eqs. 23-25).

For a point x_i with central cell b_i, every cell o = b_i + delta,
delta in {-1, 0, 1}^3, that lies inside the grid receives

    a~_{o,i} = 1/2                                       if o is the central cell
    a~_{o,i} = prod_xi 1/2 max(0, 1 - |x_xi - c_{o,xi}| / (2h))   otherwise

    alpha_{o,i} = a~_{o,i} / sum_{o' in grid} a~_{o',i}      (Eq. 24)

and V_o = sum_i alpha_{o,i} n_i (the coefficients of Eq. 23).  Cells outside
the grid are dropped before normalising (reading of the boundary case).
Non-finite points contribute nothing.
"""
from __future__ import annotations

import itertools

import numpy as np

# delta in x-fastest order: (dx, dy, dz)
OFFSETS = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                    for dx in (-1, 0, 1)], dtype=np.int64)
CENTRE_INDEX = 13


def raw_weights(points, bins, lo, h):
    """Unnormalised a~ [n, 27] and d a~/dx [n, 27, 3] (Eq. 25)."""
    p = np.asarray(points, dtype=np.float64)
    cells = bins[:, None, :] + OFFSETS[None, :, :]               # [n,27,3]
    cen = lo[None, None, :] + (cells + 0.5) * h                  # [n,27,3]
    dist = np.abs(p[:, None, :] - cen) / (2.0 * h)
    f = 0.5 * np.maximum(0.0, 1.0 - dist)                        # per-axis factor
    a = np.prod(f, axis=2)
    # derivative of each factor: -1/2 * sign(x - c) / (2h) where 1 - dist > 0
    df = np.where(1.0 - dist > 0, -0.5 * np.sign(p[:, None, :] - cen) / (2.0 * h), 0.0)
    da = np.zeros(a.shape + (3,))
    for ax in range(3):
        others = [k for k in range(3) if k != ax]
        da[:, :, ax] = df[:, :, ax] * f[:, :, others[0]] * f[:, :, others[1]]
    a[:, CENTRE_INDEX] = 0.5
    da[:, CENTRE_INDEX, :] = 0.0
    return cells, a, da


def splat_weights(points, bins, lo, h, res):
    """cells [n,27,3], alpha [n,27] (0 outside the grid), d alpha/dx [n,27,3]."""
    cells, a, da = raw_weights(points, bins, lo, h)
    inside = np.all((cells >= 0) & (cells < res), axis=2)
    a = np.where(inside, a, 0.0)
    da = np.where(inside[:, :, None], da, 0.0)
    S = a.sum(axis=1)
    dS = da.sum(axis=1)
    alpha = a / S[:, None]
    dalpha = (da - alpha[:, :, None] * dS[:, None, :]) / S[:, None, None]
    return cells, alpha, dalpha, inside


def splat(points, normals, bins, finite, lo, h, res):
    """V [res, res, res, 3] (indexed [z, y, x]) = sum_i alpha_{o,i} n_i."""
    p = np.asarray(points, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64)
    V = np.zeros((res, res, res, 3))
    keep = finite & np.all(np.isfinite(nrm), axis=1)
    if not keep.any():
        return V
    cells, alpha, _, inside = splat_weights(p[keep], bins[keep], lo, h, res)
    c = cells[inside]
    contrib = alpha[inside][:, None] * np.repeat(nrm[keep][:, None, :], 27, axis=1)[inside]
    for ax in range(3):
        np.add.at(V[..., ax], (c[:, 2], c[:, 1], c[:, 0]), contrib[:, ax])
    return V


def splat_adjoint(points, normals, bins, finite, lo, h, res, dV):
    """Given dL/dV [res,res,res,3], return (dL/dx [n,3], dL/dn [n,3])."""
    p = np.asarray(points, dtype=np.float64)
    nrm = np.asarray(normals, dtype=np.float64)
    n = p.shape[0]
    dx = np.zeros((n, 3))
    dn = np.zeros((n, 3))
    keep = finite & np.all(np.isfinite(nrm), axis=1)
    if not keep.any():
        return dx, dn
    cells, alpha, dalpha, inside = splat_weights(p[keep], bins[keep], lo, h, res)
    cc = np.clip(cells, 0, res - 1)
    g = dV[cc[..., 2], cc[..., 1], cc[..., 0], :]                 # [m,27,3]
    g = np.where(inside[..., None], g, 0.0)
    dn[keep] = np.einsum("mo,moc->mc", alpha, g)
    w = np.einsum("moc,mc->mo", g, nrm[keep])                     # n_i . dV_o
    dx[keep] = np.einsum("mo,moc->mc", w, dalpha)
    return dx, dn


def worked_example_alpha():
    """alpha for a point exactly at an interior cell centre, by offset class.

    Derived by hand from Eq. 25: centre 1/2; face neighbours (1/2)(1/2)(1/4)
    = 1/16; edge 1/32; corner 1/64; total 11/8.
    """
    out = {}
    for d in itertools.product((-1, 0, 1), repeat=3):
        k = sum(abs(v) for v in d)
        out.setdefault(k, []).append(d)
    return out
