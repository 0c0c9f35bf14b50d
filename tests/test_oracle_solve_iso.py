"""Pins for the oracle's Poisson solve (Eqs. 20-21), interpolation / iso-value
(Eq. 27), stencil normals and query interpolation."""
import numpy as np
import pytest

from oracle import iso as I
from oracle import normals as NR
from oracle import poisson as P


@pytest.mark.parametrize("n,k", [(8, (1, 0, 0)), (12, (1, 2, 0)), (10, (3, 1, 4)), (9, (8, 8, 8))])
def test_manufactured_eigenmode(n, k):
    # v_k is a discrete eigenvector of the Neumann 7-point operator with
    # eigenvalue -4 sum sin^2(pi k / 2n); a wrong boundary row breaks this.
    i = np.arange(n) + 0.5
    v = (np.cos(np.pi * k[2] * i / n)[:, None, None] * np.cos(np.pi * k[1] * i / n)[None, :, None]
         * np.cos(np.pi * k[0] * i / n)[None, None, :])
    lam = -4.0 * sum(np.sin(np.pi * kk / (2 * n)) ** 2 for kk in k)
    assert np.abs(P.laplacian(v) - lam * v).max() < 1e-12
    x = P.solve(lam * v)
    assert np.abs(x - v).max() < 1e-12


def test_laplacian_hand_rows():
    # 3^3 grid, delta at the corner: row sums and neighbour counts by hand
    chi = np.zeros((3, 3, 3))
    chi[0, 0, 0] = 1.0
    L = P.laplacian(chi)
    assert L[0, 0, 0] == -3.0                    # corner has 3 neighbours
    assert L[0, 0, 1] == 1.0 and L[0, 1, 0] == 1.0 and L[1, 0, 0] == 1.0
    chi2 = np.zeros((3, 3, 3))
    chi2[1, 1, 1] = 1.0
    assert P.laplacian(chi2)[1, 1, 1] == -6.0
    assert abs(P.laplacian(np.random.default_rng(0).random((4, 5, 6))).sum()) < 1e-12


def test_dct_solve_matches_cg_and_gauge():
    rng = np.random.default_rng(1)
    b = rng.standard_normal((10, 12, 9))
    x = P.solve(b)
    assert abs(x.sum()) < 1e-10
    assert np.abs(P.laplacian(x) - (b - b.mean())).max() < 1e-11
    assert np.abs(x - P.cg(b)).max() < 1e-10


def test_symmetry():
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal((2, 7, 6, 5))
    assert np.sum(P.laplacian(u) * v) == pytest.approx(np.sum(u * P.laplacian(v)), rel=1e-12)


def test_continuum_second_order():
    # Delta chi = -3 pi^2 cos(pi x) cos(pi y) cos(pi z) on the unit cube with
    # zero-flux walls has the solution cos cos cos; error must drop ~4x per halving.
    errs = []
    for n in (16, 32, 64):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        u = np.cos(np.pi * x)
        exact = u[:, None, None] * u[None, :, None] * u[None, None, :]
        b = -3 * np.pi ** 2 * exact * h * h            # unit-free L = h^2 Delta
        chi = P.solve(b)
        errs.append(np.abs(chi - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4


def test_trilinear_exact_on_linear_and_clamped():
    res = 7
    h = 1.0 / res
    lo = np.zeros(3)
    a = np.array([0.3, -1.2, 2.0])
    xs = (np.arange(res) + 0.5) * h
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    chi = a[0] * X + a[1] * Y + a[2] * Z + 0.7
    rng = np.random.default_rng(3)
    q = 0.5 * h + rng.random((200, 3)) * (1 - h)     # inside the node hull
    assert np.allclose(I.interpolate(chi, q, lo, h, res), q @ a + 0.7, atol=1e-13)
    # outside the hull the position is clamped per axis
    q2 = np.array([[0.0, 0.5, 0.5], [1.0, 0.5, 0.5]])
    cl = np.array([[0.5 * h, 0.5, 0.5], [1 - 0.5 * h, 0.5, 0.5]])
    assert np.allclose(I.interpolate(chi, q2, lo, h, res), cl @ a + 0.7, atol=1e-13)
    _, w, dw = I.trilinear(q2, lo, h, res)
    assert np.allclose(w.sum(1), 1.0)
    assert np.allclose(dw[:, :, 0].sum(1), 0.0)   # clamped axis: no derivative at all
    assert np.allclose(np.einsum("nc,nc->n", dw[:, :, 1], I.gather(chi, I.trilinear(q2, lo, h, res)[0])), a[1])


def test_isovalue_constant_and_linear():
    res = 6
    h = 1.0 / res
    lo = np.zeros(3)
    chi = np.full((res, res, res), 2.5)
    pts = np.random.default_rng(5).random((50, 3)) * 0.6 + 0.2
    fin = np.ones(50, bool)
    assert I.isovalue(chi, pts, fin, lo, h, res) == pytest.approx(2.5, rel=1e-15)
    xs = (np.arange(res) + 0.5) * h
    chi2 = np.broadcast_to(xs[None, None, :], (res, res, res)).copy()
    assert I.isovalue(chi2, pts, fin, lo, h, res) == pytest.approx(pts[:, 0].mean(), rel=1e-13)


def test_normals_linear_and_quadratic_exact():
    n = 6
    h = 0.1
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = 0.3 * X - 0.4 * Y + 1.2 * Z
    nrm, g, mag = NR.normals(phi, h)
    want = np.array([0.3, -0.4, 1.2]) / np.linalg.norm([0.3, -0.4, 1.2])
    assert np.allclose(np.moveaxis(nrm, 0, -1), want, atol=1e-12)
    # one-sided and central second-order stencils are exact on quadratics
    q = X * X + 2 * Y * Y - Z * Z + X * Y
    g2 = NR.gradient(q, h)
    assert np.allclose(g2[0], 2 * X + Y, atol=1e-12)
    assert np.allclose(g2[1], 4 * Y + X, atol=1e-12)
    assert np.allclose(g2[2], -2 * Z, atol=1e-12)


def test_normals_adjoint_fd():
    rng = np.random.default_rng(6)
    phi = rng.standard_normal((5, 6, 7))
    h = 0.2
    W = rng.standard_normal((3, 5, 6, 7))
    d = NR.normals_adjoint(phi, h, W)
    eps = 1e-7
    for idx in [(0, 0, 0), (2, 3, 4), (4, 5, 6), (1, 0, 6)]:
        pp = phi.copy()
        pm = phi.copy()
        pp[idx] += eps
        pm[idx] -= eps
        fd = (np.sum(NR.normals(pp, h)[0] * W) - np.sum(NR.normals(pm, h)[0] * W)) / (2 * eps)
        assert fd == pytest.approx(d[idx], rel=1e-5, abs=1e-7)
