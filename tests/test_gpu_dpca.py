"""D-PCA normal estimation (Sec. 2.1) on the GPU vs the FP64 oracle, through
the C ABI.

Bars: neighbour counts bit-exact (membership is decided in float32 on both
sides); zero normals exactly where the oracle has none; elsewhere the angle
between the (unoriented) directions within 0.1 degree wherever the oracle's
covariance has an eigen gap (lambda_1 - lambda_0) >= 1e-2 lambda_2.  Below that
gap the direction is ill-conditioned: a float32 covariance (relative error a
few 1e-6 for a few thousand terms) moves the eigenvector by about
error / gap, so those points are only checked to be unit vectors.
"""
import math

import numpy as np
import pytest

import synth
from oracle import normals_pca as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ANGLE_TOL_DEG = 0.1
GAP_REL = 1e-2
BOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)


@pytest.fixture(scope="module")
def rec():
    import __graft_entry__ as g
    g.build()
    from paper_2609_20964_gb300 import Reconstructor
    torch.cuda.set_device(0)
    r = Reconstructor(16, 200_000)
    yield r
    r.close()


def _gpu(rec, P, R, eps, bbox=BOX):
    n, c = rec.estimate_normals(torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda(), bbox, R,
                                eps, with_counts=True)
    torch.cuda.synchronize()
    return n.cpu().numpy().astype(np.float64), c.cpu().numpy()


def _compare(gn, gc, on, olam, oc):
    assert np.array_equal(gc, oc), f"counts differ at {np.nonzero(gc != oc)[0][:10]}"
    none = ~on.any(axis=1)
    assert not gn[none].any(), "GPU normal where the oracle has none"
    has = ~none
    assert np.abs(np.linalg.norm(gn[has], axis=1) - 1).max() < 1e-5
    gap = has & ((olam[:, 1] - olam[:, 0]) >= GAP_REL * olam[:, 2])
    dots = np.clip(np.abs(np.sum(gn[gap] * on[gap], axis=1)), 0, 1)
    ang = np.degrees(np.arccos(dots))
    worst = ang.max() if len(ang) else 0.0
    assert worst <= ANGLE_TOL_DEG, f"max angle {worst:.4g} deg"
    return gap.sum(), worst


def test_sh_body_cloud_matches_the_oracle(rec):
    P, _, _ = synth.sh_body_cloud(20_000, seed=31, noise=0.002)
    R = 0.05
    eps = float(np.float32(1e-3 * R))
    gn, gc = _gpu(rec, P, R, eps)
    on, olam, oc = D.dpca_normals(P.astype(np.float64), R, eps)
    checked, worst = _compare(gn, gc, on, olam, oc)
    assert checked > 0.95 * len(P)
    assert oc.min() >= 20          # neighbourhoods of the intended size


@pytest.mark.parametrize("R", [0.1])
def test_full_cloud_sampled(rec, R):
    # the 200,000-point star body at the paper's default radius R = 0.1:
    # sampled points recomputed one by one by the oracle over the whole cloud
    P, _, _ = synth.sh_body_cloud()
    eps = float(np.float32(1e-3 * R))
    gn, gc = _gpu(rec, P, R, eps)
    P64 = P.astype(np.float64)
    P32 = P.astype(np.float32)
    idx = np.random.default_rng(5).choice(len(P), 48, replace=False)
    allj = np.arange(len(P))
    on = np.zeros((len(idx), 3))
    olam = np.zeros((len(idx), 3))
    oc = np.zeros(len(idx), dtype=np.int64)
    for k, i in enumerate(idx):
        nb = D.in_ball_f32(P32, i, allj, R)
        on[k], olam[k], oc[k] = D.dpca_point(P64[i], P64[nb], eps)
    _compare(gn[idx], gc[idx], on, olam, oc)
    assert oc.min() > 1000


def test_plane_small_and_degenerate_clouds(rec):
    rng = np.random.default_rng(7)
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    Rm = q * np.sign(np.diag(r))
    uv = rng.uniform(-0.3, 0.3, (3000, 2))
    P = (np.c_[uv, np.zeros(len(uv))] @ Rm.T + 0.5).astype(np.float32)
    gn, gc = _gpu(rec, P, 0.08, 1e-4)
    ok = gc >= 3
    assert ok.mean() > 0.99
    ang = np.degrees(np.arccos(np.clip(np.abs(gn[ok] @ Rm[:, 2]), 0, 1)))
    assert ang.max() < 0.05
    on, olam, oc = D.dpca_normals(P.astype(np.float64), 0.08, float(np.float32(1e-4)))
    _compare(gn, gc, on, olam, oc)

    # n = 0: nothing to do
    e, c = rec.estimate_normals(torch.zeros((0, 3), device="cuda"), BOX, 0.1, with_counts=True)
    assert e.shape == (0, 3) and c.shape == (0,)
    # two points, duplicates, a non-finite point, a lone point
    S = np.array([[0.1, 0.1, 0.1], [0.12, 0.1, 0.1],                 # a pair: no normal
                  [0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [0.5, 0.5, 0.5],  # coincident: C = 0
                  [0.8, 0.8, 0.8], [0.81, 0.8, 0.8], [0.8, np.nan, 0.8],
                  [0.8, 0.81, 0.8], [0.9, 0.9, 0.1]], dtype=np.float32)
    gn, gc = _gpu(rec, S, 0.05, 1e-4)
    assert gc.tolist() == [2, 2, 3, 3, 3, 3, 3, 0, 3, 1]
    assert not gn[:5].any() and not gn[7].any() and not gn[9].any()
    on, olam, oc = D.dpca_normals_brute(S.astype(np.float64), 0.05, float(np.float32(1e-4)))
    _compare(gn, gc, on, olam, oc)
    assert abs(abs(gn[5, 2]) - 1) < 1e-6     # the three points span the z = 0.8 plane


def test_points_outside_the_box_and_large_cells(rec):
    P, _, _ = synth.sh_body_cloud(4000, seed=33, noise=0.002)
    R = 0.12
    eps = float(np.float32(1e-3 * R))
    on, olam, oc = D.dpca_normals(P.astype(np.float64), R, eps)
    # a box that holds part of the cloud: the rest shares the boundary cells
    half = np.array([0.3, 0.3, 0.3, 0.6, 0.6, 0.6], dtype=np.float32)
    gn, gc = _gpu(rec, P, R, eps, bbox=half)
    _compare(gn, gc, on, olam, oc)
    # a radius that puts the whole cloud in a few cells (long per-cell ranges)
    R2 = 0.7
    eps2 = float(np.float32(1e-3 * R2))
    gn, gc = _gpu(rec, P[:2500], R2, eps2)
    on, olam, oc = D.dpca_normals(P[:2500].astype(np.float64), R2, eps2)
    _compare(gn, gc, on, olam, oc)
    # a flat box (zero extent on one axis) is accepted
    flat = np.array([0, 0, 0.5, 1, 1, 0.5], dtype=np.float32)
    gn2, gc2 = _gpu(rec, P[:2500], R2, eps2, bbox=flat)
    assert np.array_equal(gc2, gc)


def test_deterministic_and_argument_checks(rec):
    from paper_2609_20964_gb300 import WgeoError
    P, _, _ = synth.sh_body_cloud(30_000, seed=34, noise=0.002)
    a = _gpu(rec, P, 0.05, 5e-5)
    b = _gpu(rec, P, 0.05, 5e-5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    Pt = torch.from_numpy(P).cuda()
    for kw in (dict(radius=0.0), dict(radius=float("nan")), dict(eps=0.0), dict(eps=-1.0),
               dict(bbox=[1, 0, 0, 0, 1, 1])):
        args = dict(bbox=BOX, radius=0.05, eps=1e-4)
        args.update(kw)
        with pytest.raises(WgeoError) as ei:
            rec.estimate_normals(Pt, args["bbox"], args["radius"], args["eps"])
        assert ei.value.code == 1
    big = torch.zeros((200_001, 3), device="cuda")
    with pytest.raises(WgeoError):
        rec.estimate_normals(big, BOX, 0.05)


def test_forward_state_survives_an_estimate(rec):
    # a normal estimate between a forward and its query leaves the forward intact
    from paper_2609_20964_gb300 import Reconstructor
    p, n = synth.sphere_cloud(2000, seed=35)
    r = Reconstructor(32, 4000)
    try:
        P = torch.from_numpy(p).cuda()
        N = torch.from_numpy(n).cuda()
        q = torch.from_numpy(synth.uniform_queries(500, 36)).cuda()
        r.reconstruct(P, N, BOX, 32)
        s0, _ = r.query(q)
        r.estimate_normals(P, BOX, 0.1)
        s1, _ = r.query(q)
        torch.cuda.synchronize()
        assert torch.equal(s0, s1)
    finally:
        r.close()
    assert math.isfinite(float(s0.abs().max()))
