"""Pins for the oracle's marching cubes (Eq. 28), exact distance (Eq. 33) and
sign (Eqs. 30, 34), and the end-to-end sphere."""
import os

import numpy as np
import pytest

import synth
from oracle import grid as G
from oracle import mc as M
from oracle import pipeline as PL
from oracle import sdf as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table_hand_cases():
    counts, tab = M.table()
    assert counts[0] == 0 and counts[255] == 0
    assert counts.max() == 5
    # one inside corner at the origin: the triangle through the x-, y- and
    # z-edges leaving corner 0, wound so its normal points away from it
    assert M.case_triangles(1) == [(0, 4, 8)]
    assert M.case_triangles(254) == [(0, 8, 4)]
    # corners 0 and 1 inside (both ends of edge 0): a quad over edges 4,5,8,9
    t = M.case_triangles(3)
    assert sorted({e for tri in t for e in tri}) == [4, 5, 8, 9] and len(t) == 2


def test_table_matches_golden():
    counts, tab = M.table()
    rows = []
    for c in range(256):
        rows.append(" ".join(str(e) for tri in M.case_triangles(c) for e in tri))
    with open(os.path.join(GOLDEN, "mc_table.txt")) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    assert lines == rows


def _random_closed_field(n, seed):
    rng = np.random.default_rng(seed)
    chi = rng.standard_normal((n, n, n))
    chi[0, :, :] = chi[-1, :, :] = 1.0
    chi[:, 0, :] = chi[:, -1, :] = 1.0
    chi[:, :, 0] = chi[:, :, -1] = 1.0
    return chi


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mesh_closed_oriented_winding(seed):
    # Random fields (outside on the domain boundary) exercise most of the 256
    # cases including the ambiguous ones.  The generalised winding number of
    # the oriented mesh must be exactly 1 at inside nodes and 0 at outside
    # nodes: that pins watertightness, orientation and the in/out rule at once.
    n = 9
    chi = _random_closed_field(n, seed)
    lo = np.zeros(3)
    h = 1.0 / n
    mesh = M.marching_cubes(chi, 0.0, lo, h)
    gid = mesh["gid"]
    # closed, consistently wound 2-chain: every directed edge is matched by as
    # many copies of its reverse (two fans of neighbouring cubes may both use
    # the same diagonal of an ambiguous shared face)
    directed = {}
    for t in gid:
        for k in range(3):
            e = (int(t[k]), int(t[(k + 1) % 3]))
            directed[e] = directed.get(e, 0) + 1
    assert all(directed.get((b, a), 0) == v for (a, b), v in directed.items())
    nodes = PL.node_xyz(np.arange(n ** 3), n, lo, h)
    w = S.winding_number(nodes, mesh["verts"])
    inside = (chi < 0.0).reshape(-1)
    assert np.allclose(w[inside], 1.0, atol=1e-6)
    assert np.allclose(w[~inside], 0.0, atol=1e-6)


def test_cases_seen_cover_table():
    seen = set()
    for seed in range(6):
        chi = _random_closed_field(9, seed)
        inside = chi < 0
        m = 8
        code = np.zeros((m, m, m), dtype=np.int64)
        for k in range(8):
            dx, dy, dz = M.CORNERS[k]
            code |= inside[dz:dz + m, dy:dy + m, dx:dx + m].astype(np.int64) << k
        seen |= set(np.unique(code).tolist())
    assert len(seen) > 200


def test_planar_field_gives_exact_plane_distance():
    n = 12
    h = 1.0 / n
    lo = np.zeros(3)
    a = np.array([0.4, 0.7, -0.3])
    a /= np.linalg.norm(a)
    xs = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    chi = a[0] * X + a[1] * Y + a[2] * Z
    c = 0.21
    mesh = M.marching_cubes(chi, c, lo, h)
    v = mesh["verts"].reshape(-1, 3)
    assert np.abs(v @ a - c).max() < 1e-14             # vertices on the plane
    nodes = PL.node_xyz(np.arange(n ** 3), n, lo, h)
    d, _ = S.exact_distance(nodes, mesh["verts"])
    sd = nodes @ a - c
    foot = nodes - sd[:, None] * a[None, :]
    inner = np.all((foot > 1.5 * h) & (foot < 1 - 1.5 * h), axis=1)
    assert inner.sum() > 200
    assert np.abs(d[inner] - np.abs(sd[inner])).max() < 1e-13
    sign = S.node_sign(chi.reshape(-1), c)
    assert np.all(sign[sd > 1e-12] == 1) and np.all(sign[sd < -1e-12] == -1)


def test_point_triangle_regions():
    a = np.array([0.0, 0.0, 0.0])
    b = np.array([1.0, 0.0, 0.0])
    c = np.array([0.0, 1.0, 0.0])
    cases = [
        ([0.2, 0.2, 0.5], 0.5),                        # face region: plane distance
        ([-1.0, -1.0, 0.0], np.sqrt(2.0)),             # vertex a
        ([2.0, 0.0, 1.0], np.sqrt(2.0)),               # vertex b
        ([0.5, -2.0, 0.0], 2.0),                       # edge ab
        ([1.0, 1.0, 0.0], np.sqrt(0.5)),               # edge bc (hypotenuse)
        ([-3.0, 0.5, 4.0], 5.0),                       # edge ca
    ]
    for p, want in cases:
        d = S.point_triangle_distance(np.array(p), a, b, c)
        assert d == pytest.approx(want, rel=1e-14)
    # against a dense barycentric lattice (an upper bound that converges)
    rng = np.random.default_rng(0)
    uu, vv = np.meshgrid(np.linspace(0, 1, 401), np.linspace(0, 1, 401))
    keep = uu + vv <= 1
    for _ in range(20):
        A, B, C = rng.standard_normal((3, 3))
        p = rng.standard_normal(3) * 2
        pts = A + uu[keep][:, None] * (B - A) + vv[keep][:, None] * (C - A)
        lattice = np.sqrt(((pts - p) ** 2).sum(1)).min()
        d = S.point_triangle_distance(p, A, B, C)
        assert d <= lattice + 1e-12 and lattice - d < 2e-3 * (1 + d)


def test_closest_point_ambiguity_cases():
    """Non-unique closest points (Eq. 33 minimisers giving different points)."""
    # two coplanar triangles sharing the edge x = 0 (y in [0, 1]) in the plane z = 0
    V = np.array([[[0, 0, 0], [0, 1, 0], [-1, 0.5, 0]],
                  [[0, 0, 0], [1, 0.5, 0], [0, 1, 0]],
                  # a parallel triangle at z = 2 above the first one
                  [[0, 0, 2], [-1, 0.5, 2], [0, 1, 2]]], dtype=np.float64)
    q = np.array([[0.0, 0.5, 0.7],      # over the shared edge: both give the same point
                  [-0.4, 0.5, 1.0],     # midway between the parallel triangles: two points
                  [-0.4, 0.5, 0.3],     # over the interior of the first, nearer to it
                  [-0.4, 0.5, 1.0 - 1e-9]])   # a hair off the medial plane: within delta
    d, _ = S.brute_force_distance(q, V)
    assert np.allclose(d, [0.7, 1.0, 0.3, 1.0 - 1e-9])
    amb = S.closest_point_ambiguous(q, V, d, delta=1e-7, sep=1e-6)
    assert amb.tolist() == [False, True, False, True]
    # with a delta below the gap the last one is unique again
    amb = S.closest_point_ambiguous(q, V, d, delta=1e-10, sep=1e-6)
    assert amb.tolist() == [False, True, False, False]


def test_pruned_search_equals_brute_force_and_parity(unit_bbox):
    p, n = synth.sphere_cloud(800, seed=11)
    rec = PL.forward_to_mesh(p, n, unit_bbox, 16)
    N = 16 ** 3
    nodes = PL.node_xyz(np.arange(N), 16, rec.lo, rec.h)
    d1, t1 = S.exact_distance(nodes, rec.mesh["verts"])
    d2, t2 = S.brute_force_distance(nodes, rec.mesh["verts"])
    assert np.array_equal(d1, d2)
    assert np.array_equal(t1, t2)
    # sign from chi equals the parity ray cast against the mesh
    inside = S.parity_inside(nodes, rec.mesh["verts"])
    assert np.array_equal(inside, rec.chi.reshape(-1) < rec.c)


def test_affine_invariance_of_phi(unit_bbox):
    # chi -> s chi + t (s > 0) moves c identically: eta, the mesh and phi are unchanged
    p, n = synth.sphere_cloud(600, seed=3)
    rec = PL.forward_to_mesh(p, n, unit_bbox, 16)
    m1 = M.marching_cubes(rec.chi, rec.c, rec.lo, rec.h)
    m2 = M.marching_cubes(3.7 * rec.chi + 11.0, 3.7 * rec.c + 11.0, rec.lo, rec.h)
    assert np.array_equal(m1["gid"], m2["gid"])
    assert np.abs(m1["verts"] - m2["verts"]).max() < 1e-12


@pytest.mark.slow
def test_sphere_64_end_to_end(unit_bbox):
    # the 4,096-point sphere at 64^3 against the analytic SDF |x - c| - r
    p, n = synth.sphere_cloud()
    rec = PL.reconstruct(p, n, unit_bbox, 64)
    h = rec.h
    X = G.node_positions(rec.lo, h, 64)
    r = np.linalg.norm(X - 0.5, axis=-1)
    ana = r - 0.3
    err = np.abs(rec.phi - ana)
    band = np.abs(ana) < 5 * h
    assert err[band].max() <= 0.5 * h
    assert err.mean() <= 0.1 * h
    assert rec.status == 0
    # Eikonal: |grad_h phi| in [0.95, 1.05] on >= 90% of nodes away from the centre
    far = r > 2 * h
    ok = (rec.gmag > 0.95) & (rec.gmag < 1.05)
    assert ok[far].mean() >= 0.9
    # sphere mesh: closed with Euler characteristic 2
    gid = rec.mesh["gid"]
    V = len(np.unique(gid))
    E = len({tuple(sorted((int(t[k]), int(t[(k + 1) % 3])))) for t in gid for k in range(3)})
    assert V - E + len(gid) == 2
