"""Pins of the parity-orientation oracle (Sec. 2.2): hand-computed detection
arrays, closed-form detection radii, brute force, and shapes whose outward
normals are known (a sphere, a thin closed slab)."""
import numpy as np

import synth
from oracle import orient as O


def _grid(n, h):
    a = np.arange(n) * h
    X, Y = np.meshgrid(a, a, indexing="ij")
    return np.c_[X.ravel(), Y.ravel()]


def test_crossings_hand_cases():
    assert O.crossings([1, 0]) == (0, 1)
    assert O.crossings([1, 1, 0, 1, 0]) == (1, 2)
    assert O.crossings([1, 0, 1, 1, 0, 0, 1, 0]) == (2, 1)
    assert O.crossings([1, 1, 1, 0]) == (0, 3)


def test_detection_radius_closed_forms_and_brute_force():
    # a square grid of spacing 1/8: nearest distance 1/8, r_d0 = 1/16 exactly
    P = np.c_[_grid(9, 0.125), np.zeros(81)]
    rd, r0 = O.detection_radius(P, 2.5)
    assert r0 == np.float32(0.0625) and rd == np.float32(0.15625)
    # an isolated point 0.75 from the grid's corner sets the maximum
    Q = np.r_[P, [[-0.75, 0.0, 0.0]]]
    rd, r0 = O.detection_radius(Q, 2.0)
    assert r0 == np.float32(0.375) and rd == np.float32(0.75)
    # random cloud with duplicates and a non-finite point: brute force in float32
    rng = np.random.default_rng(1)
    R = rng.uniform(0, 1, (300, 3)).astype(np.float32).astype(np.float64)
    R = np.r_[R, R[:3], [[np.nan, 0, 0]]]
    F = R[:-1].astype(np.float32)
    d = F[:, None, :] - F[None, :, :]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    np.fill_diagonal(d2, np.inf)
    want = np.float32(0.5) * np.sqrt(d2.min(axis=1).max())
    assert O.detection_radius(R, 2.5)[1] == want


def test_detector_equals_brute_force():
    rng = np.random.default_rng(2)
    P = rng.uniform(0, 1, (400, 3))
    det = O._Detector(P, 0.07)
    Y = rng.uniform(-0.1, 1.1, (3000, 3)).astype(np.float32)
    P32 = P.astype(np.float32)
    d = Y[:, None, :] - P32[None, :, :]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    r = np.float32(0.07)
    assert np.array_equal(det(Y), (d2 <= r * r).any(axis=1))


def test_two_planes_hand_detection_array():
    # planes z = 0 and z = 1 sampled every 1/8, so r_d = 2.5 / 16 = 5/32 and
    # ds = r_d: every probe height is exact.  From (0.5, 0.5, 0) upward the
    # probes at z = 0, 5/32 see the lower plane (5/32 exactly at r_d counts),
    # z = 30/32, 35/32 the upper one, and z = 40/32 lies beyond the widened box
    g = _grid(9, 0.125)
    P = np.r_[np.c_[g, np.zeros(len(g))], np.c_[g, np.ones(len(g))]]
    rd, _ = O.detection_radius(P)
    assert rd == np.float32(0.15625)
    det = O._Detector(P, rd)
    lo, hi = P.astype(np.float32).min(0), P.astype(np.float32).max(0)
    x = np.array([0.5, 0.5, 0.0])
    up = O.detection_array(x, [0, 0, 1], rd, det, lo, hi)
    assert up.astype(int).tolist() == [1, 1, 0, 0, 0, 0, 1, 1, 0]
    assert O.crossings(up) == (1, 2)
    down = O.detection_array(x, [0, 0, -1], rd, det, lo, hi)
    assert down.astype(int).tolist() == [1, 1, 0]
    assert O.crossings(down) == (0, 2)
    # the point's iterations: odd parity upward flips it (iteration 0), then
    # neither later criterion fires
    i = int(np.argmin(np.abs(P - x).sum(1)))
    N = np.zeros_like(P)
    N[i] = (0, 0, 1)
    out, st, _ = O.orient(P, N)
    assert out[i].tolist() == [0, 0, -1]
    assert st[i].tolist() == [1, 2, 0, 2, 1 | 8]


def test_sphere_with_random_signs_ends_outward():
    p, n = synth.sphere_cloud(3000, seed=5)
    sg = np.random.default_rng(0).choice([-1, 1], len(p)).astype(np.float32)
    out, st, rd = O.orient(p, n * sg[:, None])
    c = np.array([0.5, 0.5, 0.5])
    assert (np.sum(out * (p - c), axis=1) > 0).all()
    # outward rays cross nothing more; inward rays cross the far side once
    Nout = np.where(sg > 0, st[:, 0], st[:, 2])
    Nin = np.where(sg > 0, st[:, 2], st[:, 0])
    assert (Nout == 0).all() and (Nin == 1).all()
    # a zero normal stays zero
    z = n.copy()
    z[7] = 0
    out2, st2, _ = O.orient(p, z)
    assert not out2[7].any() and not st2[7].any()


def _thin_slab(h=0.05, t=0.09):
    """Closed box [0,1] x [0,1] x [0,t] sampled on a grid of spacing h, with
    exact outward normals."""
    g = _grid(int(round(1 / h)) + 1, h)
    pts, nrm = [], []
    pts.append(np.c_[g, np.full(len(g), t)]); nrm.append(np.tile([0, 0, 1.0], (len(g), 1)))
    pts.append(np.c_[g, np.zeros(len(g))]); nrm.append(np.tile([0, 0, -1.0], (len(g), 1)))
    s = np.arange(1, int(round(1 / h))) * h
    for zt in (t / 2,):
        for a in s:
            for v, nv in (((a, 0.0, zt), (0, -1, 0)), ((a, 1.0, zt), (0, 1, 0)),
                          ((0.0, a, zt), (-1, 0, 0)), ((1.0, a, zt), (1, 0, 0))):
                pts.append(np.array([v])); nrm.append(np.array([nv], dtype=float))
    return np.concatenate(pts), np.concatenate(nrm).astype(np.float32)


def test_thin_slab_needs_the_long_block_criterion():
    # the two faces lie within one detection block (scenario C): along an
    # inward normal the far face merges into the first block, parity alone
    # keeps it, the long-initial-block criterion flips it
    P, Nx = _thin_slab()
    faces = np.abs(Nx[:, 2]) > 0.5
    out, st, rd = O.orient(P, -Nx)
    assert rd < 0.09 < 2 * rd
    assert np.array_equal(out[faces], Nx[faces])
    assert (st[faces, 4] & 1 == 0).all()            # iteration 0 left them inward
    assert (st[faces, 4] & 2 != 0).all()            # iteration 1 flipped them
    out2, st2, _ = O.orient(P, Nx)                  # already outward: untouched
    assert np.array_equal(out2[faces], Nx[faces]) and (st2[faces, 4] == 0).all()
