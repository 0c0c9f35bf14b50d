"""Marching cubes on the node lattice (Sec. 2.4, Eq. 28).

Cubes are formed by 8 neighbouring cell centres, (res-1)^3 of them.  A node is
*inside* iff chi < c (chi grows outward because grad chi follows the outward
normals, Eq. 18); chi = c counts as outside.  On a cube edge whose endpoints
differ in class the surface vertex is q = (1 - eta) q1 + eta q2,
eta = (c - chi1) / (chi2 - chi1) (Eq. 28), with q1 the endpoint of lower index.

Lookup table.  The paper uses "the standard" table without listing it.  This
oracle derives a face-consistent table from one rule, so that neighbouring
cubes always agree on shared faces (watertight output):

* corner k of a cube sits at (k & 1, k >> 1 & 1, k >> 2 & 1);
* edge e: e = 0..3 run along x at (y, z) = (e & 1, e >> 1); e = 4..7 along y
  at (x, z) = ((e-4) & 1, (e-4) >> 1); e = 8..11 along z at (x, y) likewise;
* on each of the 6 faces the crossed edges (2 or 4) are joined by segments:
  with 2, one segment; with 4 (an ambiguous face, inside corners diagonal),
  each inside corner is cut off by the segment joining its two face edges;
* every segment is directed so that, seen from outside the cube, the inside
  corners lie to its right (reference point: the cut-off corner, or the
  centroid of the face's inside corners);
* the directed segments close into loops; loops are listed by their smallest
  edge id, each starting there, and fanned into triangles
  (l0, l_k, l_{k+1}), which then face from inside to outside.
"""
from __future__ import annotations

import numpy as np

CORNERS = np.array([(k & 1, (k >> 1) & 1, (k >> 2) & 1) for k in range(8)], dtype=np.int64)


def _edges():
    out = []
    for e in range(12):
        axis, a = divmod(e, 4)
        p = [0, 0, 0]
        others = [k for k in range(3) if k != axis]
        p[others[0]] = a & 1
        p[others[1]] = a >> 1
        q = list(p)
        q[axis] = 1
        c0 = p[0] + 2 * p[1] + 4 * p[2]
        c1 = q[0] + 2 * q[1] + 4 * q[2]
        out.append((axis, c0, c1))
    return out


EDGES = _edges()                                   # (axis, lower corner, upper corner)


def _faces():
    faces = []
    for axis in range(3):
        for side in (0, 1):
            corners = [k for k in range(8) if CORNERS[k][axis] == side]
            edges = [e for e, (ea, c0, c1) in enumerate(EDGES)
                     if ea != axis and CORNERS[c0][axis] == side]
            normal = np.zeros(3)
            normal[axis] = 1.0 if side else -1.0
            faces.append((corners, edges, normal))
    return faces


FACES = _faces()


def _edge_mid(e):
    _, c0, c1 = EDGES[e]
    return 0.5 * (CORNERS[c0] + CORNERS[c1])


def case_triangles(case: int):
    """Triangles (triples of cube edge ids) of one corner configuration."""
    inside = [(case >> k) & 1 for k in range(8)]
    crossed = [e for e, (_, c0, c1) in enumerate(EDGES) if inside[c0] != inside[c1]]
    nxt = {}
    for corners, edges, normal in FACES:
        fe = [e for e in edges if e in crossed]
        segs = []
        if len(fe) == 2:
            ins = [CORNERS[k] for k in corners if inside[k]]
            segs.append((fe[0], fe[1], np.mean(ins, axis=0)))
        elif len(fe) == 4:
            for k in corners:
                if inside[k]:
                    adj = [e for e in fe if k in (EDGES[e][1], EDGES[e][2])]
                    assert len(adj) == 2
                    segs.append((adj[0], adj[1], CORNERS[k].astype(float)))
        else:
            assert len(fe) == 0
        for a, b, ref in segs:
            pa, pb = _edge_mid(a), _edge_mid(b)
            left = np.cross(normal, pb - pa)
            if np.dot(left, ref - 0.5 * (pa + pb)) > 0:   # inside on the left: reverse
                a, b = b, a
            assert a not in nxt, "edge leaves twice"
            nxt[a] = b
    assert sorted(nxt.keys()) == sorted(crossed) and sorted(nxt.values()) == sorted(crossed)
    tris = []
    seen = set()
    for e in sorted(crossed):
        if e in seen:
            continue
        loop = [e]
        seen.add(e)
        f = nxt[e]
        while f != e:
            loop.append(f)
            seen.add(f)
            f = nxt[f]
        for k in range(1, len(loop) - 1):
            tris.append((loop[0], loop[k], loop[k + 1]))
    return tris


def build_table():
    """(counts [256], table [256, MAXT, 3] padded with -1)."""
    all_tris = [case_triangles(c) for c in range(256)]
    maxt = max(len(t) for t in all_tris)
    table = -np.ones((256, maxt, 3), dtype=np.int64)
    counts = np.zeros(256, dtype=np.int64)
    for c, t in enumerate(all_tris):
        counts[c] = len(t)
        if t:
            table[c, :len(t)] = np.array(t)
    return counts, table


_TABLE = None


def table():
    global _TABLE
    if _TABLE is None:
        _TABLE = build_table()
    return _TABLE


def cube_edge_node_offset(e):
    """Offset (dx, dy, dz) of the edge's lower endpoint within the cube, and its axis."""
    axis, c0, _ = EDGES[e]
    return CORNERS[c0], axis


def marching_cubes(chi, c, lo, h):
    """Triangles of the iso-surface chi = c.

    Returns dict with
      gid   [T, 3] global edge ids 3 * lin(lower node) + axis, lin = (z*n + y)*n + x
      verts [T, 3, 3] vertex positions (FP64)
      cube  [T] linear index of the emitting cube (cube (x,y,z) -> (z*(n-1)+y)*(n-1)+x)
    Triangles are ordered by cube index, then table order.
    """
    n = chi.shape[0]
    counts, tab = table()
    inside = chi < c
    m = n - 1
    code = np.zeros((m, m, m), dtype=np.int64)
    for k in range(8):
        dx, dy, dz = CORNERS[k]
        code |= inside[dz:dz + m, dy:dy + m, dx:dx + m].astype(np.int64) << k
    ntri = counts[code]
    cz, cy, cx = np.nonzero(ntri)
    cubes = (cz * m + cy) * m + cx
    nt = ntri[cz, cy, cx]
    # expand: one row per triangle
    rep = np.repeat(np.arange(len(cubes)), nt)
    tidx = np.arange(len(rep)) - np.repeat(np.cumsum(nt) - nt, nt)
    codes = code[cz, cy, cx][rep]
    tri_edges = tab[codes, tidx]                                  # [T,3] cube edge ids
    base = np.stack([cx[rep], cy[rep], cz[rep]], axis=1)          # [T,3]
    offs = np.array([cube_edge_node_offset(e)[0] for e in range(12)])
    axes = np.array([cube_edge_node_offset(e)[1] for e in range(12)])
    node = base[:, None, :] + offs[tri_edges]                     # [T,3,3]
    axis = axes[tri_edges]                                        # [T,3]
    lin = (node[..., 2] * n + node[..., 1]) * n + node[..., 0]
    gid = 3 * lin + axis
    verts = edge_vertices(chi, c, lo, h, gid)
    return {"gid": gid, "verts": verts, "cube": cubes[rep], "n": n}


def edge_endpoints(gid, n):
    """Lower node (x,y,z), axis and upper node of global edge ids."""
    lin, axis = np.divmod(gid, 3)
    z, rem = np.divmod(lin, n * n)
    y, x = np.divmod(rem, n)
    p = np.stack([x, y, z], axis=-1)
    q = p.copy()
    for a in range(3):
        q[..., a] += (axis == a)
    return p, axis, q


def edge_eta(chi, c, gid):
    n = chi.shape[0]
    p, axis, q = edge_endpoints(gid, n)
    c1 = chi[p[..., 2], p[..., 1], p[..., 0]]
    c2 = chi[q[..., 2], q[..., 1], q[..., 0]]
    return (c - c1) / (c2 - c1), c1, c2, p, axis


def edge_vertices(chi, c, lo, h, gid):
    eta, _, _, p, axis = edge_eta(chi, c, gid)
    pos = lo + (p + 0.5) * h
    off = np.zeros(pos.shape)
    for a in range(3):
        off[..., a] = np.where(axis == a, eta * h, 0.0)
    return pos + off
