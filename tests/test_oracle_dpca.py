"""Pins of the D-PCA normal-estimation oracle (Sec. 2.1) by closed forms,
symmetry and brute force."""
import numpy as np

from oracle import normals_pca as D


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


def test_plane_gives_the_plane_normal():
    rng = np.random.default_rng(1)
    R = _rotation(rng)
    uv = rng.uniform(-1, 1, (400, 2))
    P = np.c_[uv, np.zeros(len(uv))] @ R.T + np.array([0.3, -0.2, 0.5])
    n, lam, cnt = D.dpca_normals(P, radius=0.3, eps=1e-4)
    ok = cnt >= 3
    assert ok.mean() > 0.95
    assert np.abs(np.abs(n[ok] @ R[:, 2]) - 1.0).max() < 1e-10
    assert np.abs(lam[ok, 0]).max() < 1e-14


def test_symmetric_cap_gives_the_radial_direction():
    # the pole of a sphere with rings of points at equal azimuth steps: the
    # weighted covariance is symmetric about the axis, so its smallest
    # eigenvector is the axis itself
    r = 0.4
    pts = [[0.0, 0.0, r]]
    for th in (0.1, 0.2, 0.3):
        for k in range(7):
            ph = 2 * np.pi * k / 7 + th
            pts.append([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)])
    P = np.array(pts)
    n, lam, cnt = D.dpca_point(P[0], P, eps=1e-3)
    assert cnt == len(P)
    assert abs(abs(n[2]) - 1.0) < 1e-12
    assert lam[0] < lam[1] - 1e-6


def test_hand_computed_cross():
    # x_i = 0 and four neighbours at unit distance on the x and y axes:
    # centroid 0, C = 2 / ((1 + eps) W) diag(1, 1, 0), W = 1/eps + 4/(1 + eps)
    eps = 1e-3
    P = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]], dtype=float)
    n, lam, cnt = D.dpca_point(P[0], P, eps)
    W = 1 / eps + 4 / (1 + eps)
    c = 2 / ((1 + eps) * W)
    assert cnt == 5
    assert abs(abs(n[2]) - 1) < 1e-14
    assert np.allclose(lam, [0.0, c, c], atol=1e-15, rtol=1e-12)


def test_kdtree_equals_brute_force_and_equivariance():
    rng = np.random.default_rng(2)
    P = rng.standard_normal((300, 3)) * np.array([1.0, 0.6, 0.05])
    a = D.dpca_normals(P, 0.5, 1e-4)
    b = D.dpca_normals_brute(P, 0.5, 1e-4)
    assert np.array_equal(a[2], b[2])
    # where a normal exists and is unique (a gap below the second eigenvalue)
    gap = (a[2] >= 3) & ((a[1][:, 1] - a[1][:, 0]) > 1e-6 * (a[1][:, 2] + 1e-300))
    assert gap.mean() > 0.9
    assert np.allclose(np.abs(np.sum(a[0][gap] * b[0][gap], axis=1)), 1.0, atol=1e-12)
    assert not a[0][a[2] < 3].any()
    R = _rotation(rng)
    c = D.dpca_normals(P @ R.T + 1.0, 0.5, 1e-4)
    assert np.array_equal(a[2], c[2])
    dots = np.abs(np.sum((a[0] @ R.T)[gap] * c[0][gap], axis=1))
    assert np.abs(dots - 1).max() < 1e-8


def test_degenerate_neighbourhoods():
    # fewer than 3 points: no normal; collinear points: a zero-variance plane
    P = np.array([[0, 0, 0], [0.1, 0, 0], [5, 5, 5]], dtype=float)
    n, lam, cnt = D.dpca_normals(P, 0.2, 1e-4)
    assert cnt.tolist() == [2, 2, 1]
    assert not n.any()
    L = np.c_[np.linspace(0, 1, 20), np.zeros(20), np.zeros(20)]
    n, lam, cnt = D.dpca_normals(L, 0.3, 1e-4)
    assert np.abs(lam[:, :2]).max() < 1e-14     # two zero eigenvalues: direction not unique
    assert np.abs(n[:, 0]).max() < 1e-12         # but orthogonal to the line


def test_covariance_by_the_moment_identity():
    # C = E_w[y y^T] - E_w[y] E_w[y]^T (y = x_j - x_i, weighted means): an
    # independent route to the centred covariance, on a cloud whose weighted
    # centroid is far from the query point
    rng = np.random.default_rng(3)
    x = np.zeros(3)
    X = np.r_[[x], rng.uniform(0.2, 1.0, (30, 3)) * np.array([1.0, 0.7, 0.2])]
    eps = 0.5
    n, lam, cnt = D.dpca_point(x, X, eps)
    y = X - x
    w = 1.0 / (np.linalg.norm(y, axis=1) + eps)
    m = (w[:, None] * y).sum(0) / w.sum()
    C = np.einsum("j,ja,jb->ab", w, y, y) / w.sum() - np.outer(m, m)
    lam2, V2 = np.linalg.eigh(C)
    assert np.allclose(lam, lam2, rtol=1e-10, atol=1e-14)
    assert abs(abs(n @ V2[:, 0]) - 1) < 1e-10
    # the uncentred moment would point elsewhere: the pin can tell them apart
    lam3, V3 = np.linalg.eigh(np.einsum("j,ja,jb->ab", w, y, y) / w.sum())
    assert abs(abs(n @ V3[:, 0]) - 1) > 1e-3


def test_float32_membership_matches_the_ball_away_from_its_boundary():
    # the float32 test and the FP64 ball differ only for pairs whose distance
    # is within a few float32 ulps of R; planted pairs at R(1 -+ 1e-5) are
    # decided the same by both, a pair at exactly R is inside for both
    rng = np.random.default_rng(4)
    P = rng.uniform(-1, 1, (400, 3)).astype(np.float32).astype(np.float64)
    R = 0.25
    a = D.dpca_normals(P, R, 1e-4)
    b = D.dpca_normals(P, R, 1e-4, exact_ball=True)
    d = np.linalg.norm(P[:, None, :] - P[None, :, :], axis=2)
    near = (np.abs(d - R) < 1e-6 * R).any(axis=1)
    assert np.array_equal(a[2][~near], b[2][~near])
    P2 = np.array([[0, 0, 0], [R * (1 - 1e-5), 0, 0], [0, R * (1 + 1e-5), 0], [0, 0, 0.25]])
    c = D.dpca_normals_brute(P2, R, 1e-4)
    assert c[2].tolist() == [3, 2, 1, 2]
    # a non-finite point joins no neighbourhood and has no normal
    P3 = np.r_[P[:50], [[np.nan, 0, 0]]]
    e = D.dpca_normals(P3, R, 1e-4)
    f = D.dpca_normals(P[:50], R, 1e-4)
    assert np.array_equal(e[2][:50], f[2]) and e[2][50] == 0 and not e[0][50].any()
