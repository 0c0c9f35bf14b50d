"""Exact signed distance to the extracted surface at arbitrary query points
(Sec. 2.4, Eqs. 29-34, evaluated off the grid).  Test infrastructure only:
the CUDA path never imports it.

  d(q)    = min_k d(q, T_k)                         (Eq. 33, every triangle)
  s(q)    = -1 if a ray from q crosses the surface an odd number of times,
            +1 otherwise                            (Eq. 34, parity test)
  phi(q)  = s(q) d(q)                               (Eq. 30)
  grad(q) = s(q) (q - y) / d(q), y the closest surface point: the gradient of
            phi wherever the closest point is unique and d > 0.

The distance is the k-d-tree-pruned exact search of `sdf.exact_distance`,
the sign `sdf.parity_inside` (a generic ray direction, re-cast on degenerate
hits).  Where d = 0 the gradient is reported as zero.
"""
from __future__ import annotations

import numpy as np

from . import sdf as S


def query_exact(q, verts):
    """(phi [m], grad [m, 3], closest triangle [m]) at the query points q."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, 3)
    V = np.asarray(verts, dtype=np.float64)
    d, tri = S.exact_distance(q, V)
    inside = S.parity_inside(q, V)
    s = np.where(inside, -1.0, 1.0)
    ok = tri >= 0
    y = np.zeros_like(q)
    if ok.any():
        y[ok], _ = S.closest_point_triangle(q[ok], V[tri[ok], 0], V[tri[ok], 1], V[tri[ok], 2])
    grad = np.zeros_like(q)
    pos = ok & (d > 0)
    grad[pos] = s[pos, None] * (q[pos] - y[pos]) / d[pos, None]
    return s * d, grad, tri
