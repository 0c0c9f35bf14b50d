"""Pins for the oracle's restricted forward and the shape-parameter gradient
(Sec. 2.5, last paragraph; Sec. 3.3; loss reading R11):

* phi, distance and closest triangle evaluated only at chosen nodes equal the
  full-grid forward's values there (NaN / -1 elsewhere), with and without a
  process pool;
* the theta-gradient of the query loss (adjoint chain + generator VJP) equals
  central finite differences of the FP64 loss along several directions, with
  the central cells frozen (reading R12)."""
import numpy as np
import pytest

import synth
from oracle import pipeline as PL
from oracle import sdf as S
from oracle import shape_opt as SO

BBOX = np.array([0, 0, 0, 1, 1, 1], np.float32)


def test_restricted_forward_equals_full_grid():
    res = 14
    p, n = synth.sphere_cloud(600, seed=31)
    full = PL.reconstruct(p, n, BBOX, res, with_normals=False)
    lin = np.random.default_rng(2).choice(res ** 3, 500, replace=False)
    part = PL.reconstruct_at_nodes(p, n, BBOX, res, lin)
    assert np.array_equal(part.phi.reshape(-1)[lin], full.phi.reshape(-1)[lin])
    assert np.array_equal(part.tri.reshape(-1)[lin], full.tri.reshape(-1)[lin])
    other = np.setdiff1d(np.arange(res ** 3), lin)
    assert np.isnan(part.phi.reshape(-1)[other]).all()
    assert (part.tri.reshape(-1)[other] == -1).all()
    # query corners: every trilinear corner of every query is among them
    q = synth.uniform_queries(300, seed=4)
    cn = PL.query_corner_nodes(q, res, full.lo, full.h)
    from oracle import iso as I
    corners, _, _ = I.trilinear(q.astype(np.float64), full.lo, full.h, res)
    want = np.unique(((corners[..., 2] * res + corners[..., 1]) * res + corners[..., 0]).reshape(-1))
    assert np.array_equal(cn, want)


def test_distance_pool_equals_serial():
    res = 12
    p, n = synth.sphere_cloud(400, seed=32)
    rec = PL.forward_to_mesh(p, n, BBOX, res)
    nodes = PL.node_xyz(np.arange(res ** 3), res, rec.lo, rec.h)
    d1, t1 = S.exact_distance(nodes, rec.mesh["verts"])
    d2, t2 = S.exact_distance_pool(nodes, rec.mesh["verts"], workers=2, parts=8)
    assert np.array_equal(d1, d2) and np.array_equal(t1, t2)


@pytest.mark.slow
def test_theta_gradient_matches_central_fd():
    # a degree-2 body (9 coefficients), 3000 fixed directions, 18^3 grid,
    # 2000 queries, target from other coefficients of the same family
    res = 18
    rng = np.random.default_rng(7)
    dirs = synth.uniform_dirs(3000, rng)
    th0 = np.zeros(9)
    th0[0] = 0.05
    th0[1:] = rng.normal(0, 0.02, 8)
    tht = th0 + rng.normal(0, 0.02, 9)
    q = synth.uniform_queries(2000, seed=8).astype(np.float64)
    pt, nt = SO.sh_cloud(tht, dirs, float32=False)
    phi_t, _ = SO.phi_at_queries(pt, nt, q, BBOX, res)
    p0, n0 = SO.sh_cloud(th0, dirs, float32=False)
    phi0, rec0 = SO.phi_at_queries(p0, n0, q, BBOX, res)
    assert SO.loss(phi0, phi_t) > 0
    dth, dp, dn = SO.theta_gradient(th0, dirs, rec0, q, SO.loss_seeds(phi0, phi_t))
    assert dp.shape == p0.shape and dn.shape == n0.shape
    eps = 1e-6
    for v in (dth / np.linalg.norm(dth), np.eye(9)[0], np.eye(9)[4], rng.standard_normal(9) / 3):
        Ls = []
        for sgn in (1.0, -1.0):
            pp, nn = SO.sh_cloud(th0 + sgn * eps * v, dirs, float32=False)
            ph, _ = SO.phi_at_queries(pp, nn, q, BBOX, res, frozen_bins=rec0.bins)
            Ls.append(SO.loss(ph, phi_t))
        fd = (Ls[0] - Ls[1]) / (2 * eps)
        assert fd == pytest.approx(float(dth @ v), rel=1e-4, abs=1e-4 * np.linalg.norm(dth))


def test_stored_c3_differences_agree_with_the_stored_adjoint():
    """The full-size differentiable workload (128^3, 100k points, 500k
    queries) as stored by tests/golden/make_c3_fd.py: the oracle's adjoint
    gradient along each stored direction equals the central finite difference
    of its own loss (step 1e-4, central cells frozen) within 1e-2, the
    method's stated gradient tolerance against differences."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c3_theta_fd.json")) as f:
        d = json.load(f)
    g = np.asarray(d["oracle_dtheta"])
    assert g.shape == (49,) and d["eps"] == 1e-4
    for name, v, fd in zip(d["names"], d["directions"], d["fd"]):
        ad = float(g @ np.asarray(v))
        assert abs(ad - fd) <= 1e-2 * abs(fd), (name, ad, fd)
