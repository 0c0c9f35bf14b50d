"""Exact signed distance to the extracted surface (Sec. 2.4, Eqs. 29-34).

Distance (Eq. 33): d(q) = min over all triangles T_k of d(q, T_k).  The
point-to-triangle distance follows the paper's description: project q on the
triangle's plane; if the projection is inside the triangle, the distance is
the plane distance; otherwise it is the smallest distance to the three edges
(segments, which include the vertices).

Search: exact, never approximate.  The upper bound U(q) = distance to the
nearest triangle centroid (a point of the surface) is found with a k-d tree;
every triangle within U of q has its centroid within U + rho of q, rho the
largest centroid-to-vertex radius, so the candidates returned by a ball query
of radius U + rho contain the minimiser.  Brute force over all triangles is
kept for the small cross-checks.

Sign (Eq. 30, 34): at grid nodes the surface separates nodes with chi < c
(inside, sign -1) from the rest (outside, +1) by construction; the paper's
parity ray cast (Sec. 2.2 crossing-number rule applied to the mesh) is
implemented here as well, to check that both agree.

Ties between triangles resolve to the smaller distance, then the smaller
triangle index.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def _closest_on_segment(p, a, b):
    ab = b - a
    L2 = np.sum(ab * ab, axis=-1)
    t = np.where(L2 > 0, np.sum((p - a) * ab, axis=-1) / np.where(L2 > 0, L2, 1.0), 0.0)
    t = np.clip(t, 0.0, 1.0)
    return a + t[..., None] * ab, t


def closest_point_triangle(p, a, b, c):
    """Closest point y on triangle (a,b,c) to p and its barycentrics (wa, wb, wc).

    Arrays broadcast over leading dimensions, last dimension 3.
    """
    p, a, b, c = np.broadcast_arrays(p, a, b, c)
    ab = b - a
    ac = c - a
    ap = p - a
    # projection on the plane: solve [ab.ab ab.ac; ab.ac ac.ac] [v w] = [ab.ap ac.ap]
    d00 = np.sum(ab * ab, -1)
    d01 = np.sum(ab * ac, -1)
    d11 = np.sum(ac * ac, -1)
    r0 = np.sum(ab * ap, -1)
    r1 = np.sum(ac * ap, -1)
    det = d00 * d11 - d01 * d01
    ok = det > 1e-300
    sdet = np.where(ok, det, 1.0)
    v = (d11 * r0 - d01 * r1) / sdet
    w = (d00 * r1 - d01 * r0) / sdet
    u = 1.0 - v - w
    inside = ok & (u >= 0) & (v >= 0) & (w >= 0)
    y_face = a + v[..., None] * ab + w[..., None] * ac
    # edges
    y_ab, t_ab = _closest_on_segment(p, a, b)
    y_bc, t_bc = _closest_on_segment(p, b, c)
    y_ca, t_ca = _closest_on_segment(p, c, a)
    d_ab = np.sum((p - y_ab) ** 2, -1)
    d_bc = np.sum((p - y_bc) ** 2, -1)
    d_ca = np.sum((p - y_ca) ** 2, -1)
    best = np.argmin(np.stack([d_ab, d_bc, d_ca], -1), axis=-1)
    y_edge = np.where((best == 0)[..., None], y_ab, np.where((best == 1)[..., None], y_bc, y_ca))
    bary_edge = np.stack([
        np.where(best == 0, 1 - t_ab, np.where(best == 2, t_ca, 0.0)),
        np.where(best == 0, t_ab, np.where(best == 1, 1 - t_bc, 0.0)),
        np.where(best == 1, t_bc, np.where(best == 2, 1 - t_ca, 0.0)),
    ], -1)
    y = np.where(inside[..., None], y_face, y_edge)
    bary = np.where(inside[..., None], np.stack([u, v, w], -1), bary_edge)
    return y, bary


def point_triangle_distance(p, a, b, c):
    y, _ = closest_point_triangle(p, a, b, c)
    return np.sqrt(np.sum((p - y) ** 2, -1))


def brute_force_distance(nodes, verts):
    """(d [N], tri [N]) by testing every triangle against every node."""
    N = nodes.shape[0]
    d = np.full(N, np.inf)
    tri = np.full(N, -1, dtype=np.int64)
    for t in range(verts.shape[0]):
        dt = point_triangle_distance(nodes, verts[t, 0], verts[t, 1], verts[t, 2])
        better = dt < d
        d = np.where(better, dt, d)
        tri = np.where(better, t, tri)
    return d, tri


def exact_distance(nodes, verts, chunk: int = 16384):
    """Exact nearest-triangle distance and index for every node (k-d tree pruned)."""
    N = nodes.shape[0]
    T = verts.shape[0]
    d = np.full(N, np.inf)
    tri = np.full(N, -1, dtype=np.int64)
    if T == 0 or N == 0:
        return d, tri
    cent = verts.mean(axis=1)
    rho = float(np.max(np.linalg.norm(verts - cent[:, None, :], axis=2)))
    tree = cKDTree(cent)
    for s in range(0, N, chunk):
        q = nodes[s:s + chunk]
        U, _ = tree.query(q)
        cands = tree.query_ball_point(q, U * (1 + 1e-12) + rho + 1e-15)
        lens = np.array([len(cc) for cc in cands])
        flat = np.concatenate([np.asarray(cc, dtype=np.int64) for cc in cands])
        owner = np.repeat(np.arange(len(q)), lens)
        # stable order inside each node: ascending triangle index
        order = np.lexsort((flat, owner))
        flat = flat[order]
        owner = owner[order]
        dd = point_triangle_distance(q[owner], verts[flat, 0], verts[flat, 1], verts[flat, 2])
        starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
        mind = np.minimum.reduceat(dd, starts)
        # smallest triangle index among the minimisers
        is_min = dd == mind[owner]
        big = np.where(is_min, flat, np.iinfo(np.int64).max)
        argt = np.minimum.reduceat(big, starts)
        d[s:s + chunk] = mind
        tri[s:s + chunk] = argt
    return d, tri


def _exact_distance_part(args):
    nodes, verts = args
    return exact_distance(nodes, verts)


def exact_distance_pool(nodes, verts, workers: int = 1, parts: int = 64, pool=None):
    """exact_distance, with the nodes split into contiguous parts evaluated by
    a pool of `workers` processes (started with "spawn", so the pool may be
    created in a process that already uses a GPU), or by `pool` when given.
    Every node's result is computed by exact_distance itself; only the work is
    divided."""
    N = nodes.shape[0]
    if (workers <= 1 and pool is None) or N < 4 * parts:
        return exact_distance(nodes, verts)
    bounds = np.linspace(0, N, parts + 1).astype(np.int64)
    jobs = [(nodes[bounds[i]:bounds[i + 1]], verts) for i in range(parts)]
    if pool is not None:
        out = pool.map(_exact_distance_part, jobs, chunksize=1)
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as own:
            out = own.map(_exact_distance_part, jobs, chunksize=1)
    return np.concatenate([o[0] for o in out]), np.concatenate([o[1] for o in out])


def node_sign(chi, c):
    return np.where(chi >= c, 1.0, -1.0)


RAY_DIR = np.array([0.5773, 0.5774, 0.5775]) / np.linalg.norm([0.5773, 0.5774, 0.5775])


def parity_inside(nodes, verts, direction=RAY_DIR, eps=1e-10):
    """Crossing-number inside test against the triangle mesh (odd = inside).

    Degenerate hits (on an edge or vertex, or at the origin) are re-cast with a
    perturbed direction.
    """
    out = np.zeros(nodes.shape[0], dtype=bool)
    a, b, c = verts[:, 0], verts[:, 1], verts[:, 2]
    e1 = b - a
    e2 = c - a
    rng = np.random.default_rng(12345)
    for i, q in enumerate(nodes):
        dvec = direction
        for _attempt in range(20):
            pvec = np.cross(dvec, e2)
            det = np.sum(e1 * pvec, axis=1)
            good = np.abs(det) > 1e-300
            inv = np.where(good, 1.0 / np.where(good, det, 1.0), 0.0)
            tvec = q - a
            u = np.sum(tvec * pvec, axis=1) * inv
            qvec = np.cross(tvec, e1)
            v = (qvec @ dvec) * inv
            t = np.sum(e2 * qvec, axis=1) * inv
            hit = good & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
            near = good & (t > -eps) & (
                (np.abs(u) < eps) | (np.abs(v) < eps) | (np.abs(1 - u - v) < eps) | (np.abs(t) < eps)
            ) & (u > -eps) & (v > -eps) & (u + v < 1 + eps)
            if not near.any():
                out[i] = bool(hit.sum() % 2)
                break
            dvec = dvec + 1e-3 * rng.standard_normal(3)
            dvec /= np.linalg.norm(dvec)
    return out


def winding_number(points, verts):
    """Generalised winding number of the oriented mesh at each point."""
    w = np.zeros(points.shape[0])
    for i, q in enumerate(points):
        A = verts[:, 0] - q
        B = verts[:, 1] - q
        C = verts[:, 2] - q
        la, lb, lc = (np.linalg.norm(X, axis=1) for X in (A, B, C))
        num = np.sum(A * np.cross(B, C), axis=1)
        den = (la * lb * lc + np.sum(A * B, 1) * lc + np.sum(A * C, 1) * lb
               + np.sum(B * C, 1) * la)
        w[i] = np.sum(2.0 * np.arctan2(num, den)) / (4 * np.pi)
    return w


def closest_point_ambiguous(nodes, verts, d, delta, sep, chunk: int = 2048):
    """True where the closest surface point of a node is not unique.

    A node is ambiguous when some triangle lies within ``delta`` of the
    minimum distance ``d`` (Eq. 33) but its closest point is more than ``sep``
    away from the closest point of the minimising triangle.  There the
    distance is not differentiable in the vertices (the node sits on, or
    within rounding of, the medial axis of the mesh), so two exact
    implementations may legitimately pick different triangles and obtain
    different vertex gradients.  Triangles sharing the closest edge or vertex
    give the same point and do not count.  Exact, k-d tree pruned: a triangle
    with centroid m and centroid radius r_t can only be within d + delta of q
    if |q - m| <= d + delta + r_t.
    """
    N = nodes.shape[0]
    amb = np.zeros(N, dtype=bool)
    if verts.shape[0] == 0 or N == 0:
        return amb
    cent = verts.mean(axis=1)
    rad = np.max(np.linalg.norm(verts - cent[:, None, :], axis=2), axis=1)
    rho = float(rad.max())
    tree = cKDTree(cent)
    for s in range(0, N, chunk):
        q = nodes[s:s + chunk]
        dq = d[s:s + chunk]
        cands = tree.query_ball_point(q, dq + delta + rho + 1e-15)
        lens = np.array([len(cc) for cc in cands])
        if lens.sum() == 0:
            continue
        flat = np.concatenate([np.asarray(cc, dtype=np.int64) for cc in cands])
        owner = np.repeat(np.arange(len(q)), lens)
        keep = np.linalg.norm(q[owner] - cent[flat], axis=1) <= dq[owner] + delta + rad[flat] + 1e-15
        flat, owner = flat[keep], owner[keep]
        y, _ = closest_point_triangle(q[owner], verts[flat, 0], verts[flat, 1], verts[flat, 2])
        dd = np.sqrt(np.sum((q[owner] - y) ** 2, -1))
        near = dd <= dq[owner] + delta
        # the closest point of the minimiser, per node
        best = np.full(len(q), np.inf)
        np.minimum.at(best, owner, dd)
        is_best = dd == best[owner]
        ybest = np.zeros((len(q), 3))
        ybest[owner[is_best]] = y[is_best]
        far = near & (np.linalg.norm(y - ybest[owner], axis=1) > sep)
        amb[s:s + chunk] |= np.bincount(owner[far], minlength=len(q)).astype(bool)
    return amb
