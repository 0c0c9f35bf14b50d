"""Pins of the exact off-grid signed distance (Sec. 2.4, Eqs. 29-34 at
arbitrary points): a sphere mesh against the analytic distance, the grid
nodes of a reconstruction against the node definition (sign from the
indicator), central differences of the gradient, and the winding number."""
import numpy as np

import synth
from oracle import pipeline as OP
from oracle import query_exact as QE
from oracle import sdf as S


def _icosphere(level, r=0.3, c=(0.5, 0.5, 0.5)):
    t = (1 + 5 ** 0.5) / 2
    V = [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]]
    F = [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
         [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5], [2, 4, 11],
         [6, 2, 10], [8, 6, 7], [9, 8, 1]]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    for _ in range(level):
        mid = {}
        G = []
        for a, b, cc in F:
            ids = []
            for u, w in ((a, b), (b, cc), (cc, a)):
                key = (min(u, w), max(u, w))
                if key not in mid:
                    m = V[u] + V[w]
                    V.append(m / np.linalg.norm(m))
                    mid[key] = len(V) - 1
                ids.append(mid[key])
            G += [[a, ids[0], ids[2]], [b, ids[1], ids[0]], [cc, ids[2], ids[1]], ids]
        F = G
    V = np.array(V) * r + np.asarray(c)
    return V[np.array(F)]


def test_sphere_mesh_against_the_analytic_distance():
    # vertices on the sphere, flat faces inside it: the surface lies between
    # the sphere and the concentric sphere of radius r - gap, gap = r minus the
    # smallest distance from the centre to a face plane
    tris = _icosphere(3)
    r = 0.3
    edge = np.max(np.linalg.norm(tris[:, 0] - tris[:, 1], axis=1))
    nf = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    nf /= np.linalg.norm(nf, axis=1)[:, None]
    gap = r - np.min(np.abs(np.sum(nf * (tris[:, 0] - 0.5), axis=1))) + 1e-12
    rng = np.random.default_rng(0)
    q = rng.uniform(0.0, 1.0, (400, 3))
    phi, grad, tri = QE.query_exact(q, tris)
    a = np.linalg.norm(q - 0.5, axis=1) - r
    # the faces lie between the sphere and the sphere shrunk by gap, on both
    # sides: a <= phi <= a + gap
    assert np.all(phi >= a - 1e-12) and np.all(phi <= a + gap)
    clear = np.abs(a) > gap                      # outside the sliver between faces and sphere
    assert (np.sign(phi[clear]) == np.sign(a[clear])).all()
    # far from the surface the gradient is the radial direction, up to the facet angle
    far = np.abs(a) > 0.05
    radial = (q - 0.5) / np.linalg.norm(q - 0.5, axis=1)[:, None]
    cosang = np.sum(grad[far] * radial[far], axis=1)
    assert cosang.min() > np.cos(np.arcsin(edge / (2 * r)) + 0.2)


def test_grid_nodes_reproduce_the_node_definition():
    # at the nodes of a reconstruction, the parity sign equals the indicator
    # class and the distance equals the node search: phi matches the grid
    p, n = synth.sphere_cloud(1500, seed=21)
    rec = OP.reconstruct(p, n, np.array([0, 0, 0, 1, 1, 1], float), 16, with_normals=False)
    verts = rec.mesh["verts"]
    phi_grid = rec.phi
    res = 16
    h = 1.0 / res
    idx = np.random.default_rng(3).choice(res ** 3, 300, replace=False)
    k, j, i = np.unravel_index(idx, (res, res, res))
    nodes = np.c_[(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h]
    phi, _, _ = QE.query_exact(nodes, verts)
    assert np.allclose(phi, phi_grid.reshape(-1)[idx], rtol=0, atol=1e-12)


def test_gradient_matches_central_differences():
    tris = _icosphere(2, r=0.25)
    rng = np.random.default_rng(5)
    q = rng.uniform(0.1, 0.9, (60, 3))
    phi, grad, _ = QE.query_exact(q, tris)
    amb = S.closest_point_ambiguous(q, tris, np.abs(phi), 1e-6, 1e-4)
    keep = (~amb) & (np.abs(phi) > 1e-3)
    hstep = 1e-6
    fd = np.zeros_like(q)
    for a in range(3):
        e = np.zeros(3)
        e[a] = hstep
        fd[:, a] = (QE.query_exact(q + e, tris)[0] - QE.query_exact(q - e, tris)[0]) / (2 * hstep)
    assert keep.sum() > 40
    assert np.abs(fd[keep] - grad[keep]).max() < 1e-6
    assert np.allclose(np.linalg.norm(grad[keep], axis=1), 1.0)


def test_sign_agrees_with_the_winding_number():
    tris = _icosphere(2)
    rng = np.random.default_rng(6)
    q = rng.uniform(0, 1, (200, 3))
    phi, _, _ = QE.query_exact(q, tris)
    w = S.winding_number(q, tris)
    assert np.array_equal(phi < 0, w > 0.5)
