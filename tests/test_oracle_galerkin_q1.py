"""Pins of the unlumped trilinear Galerkin operator (Sec. 2.3, Eqs. 20-22 and
26 with the trilinear hat of Eq. 16): the stencil and the right-hand side
against direct numerical quadrature of the defining integrals, the DCT
eigenmodes in closed form, the lumping identity with the 7-point operator,
symmetry, the Neumann null space and the solve."""
import numpy as np

from oracle import divergence as D
from oracle import galerkin_q1 as Q
from oracle import poisson as P

# Gauss-Legendre nodes on [0, 1]: exact for the piecewise polynomials below
_GX, _GW = np.polynomial.legendre.leggauss(4)
_GX = 0.5 * (_GX + 1.0)
_GW = 0.5 * _GW


def _hat(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


def _dhat(t):
    return np.where(np.abs(t) < 1.0, -np.sign(t), 0.0)


def _cells_quadrature(f):
    """Integral of f(x, y, z) over [-1, 1]^3 (unit cells, 4^3 Gauss points each)."""
    tot = 0.0
    for a in (-1, 0):
        for b in (-1, 0):
            for c in (-1, 0):
                X, Y, Z = np.meshgrid(a + _GX, b + _GX, c + _GX, indexing="ij")
                Wt = _GW[:, None, None] * _GW[None, :, None] * _GW[None, None, :]
                tot += float(np.sum(Wt * f(X, Y, Z)))
    return tot


def test_interior_stencil_is_the_galerkin_integral():
    # A_{p,o} = int grad F_p . grad F_o with F_p centred at 0 and F_o at delta
    # (h = 1): against L27 = -A applied to an impulse in the interior
    n = 7
    e = np.zeros((n, n, n))
    e[3, 3, 3] = 1.0
    col = Q.laplacian27(e)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                def f(X, Y, Z):
                    return (_dhat(X) * _dhat(X - dx) * _hat(Y) * _hat(Y - dy) * _hat(Z) * _hat(Z - dz)
                            + _hat(X) * _hat(X - dx) * _dhat(Y) * _dhat(Y - dy) * _hat(Z) * _hat(Z - dz)
                            + _hat(X) * _hat(X - dx) * _hat(Y) * _hat(Y - dy) * _dhat(Z) * _dhat(Z - dz))
                a_po = _cells_quadrature(f)
                assert abs(-col[3 + dz, 3 + dy, 3 + dx] - a_po) < 1e-12, (dx, dy, dz, a_po)
    assert abs(col[3, 3, 3] + 8.0 / 3.0) < 1e-14
    assert abs(col[3, 3, 4]) < 1e-14 and abs(col[3, 4, 4] - 1.0 / 6.0) < 1e-14
    assert abs(col[4, 4, 4] - 1.0 / 12.0) < 1e-14


def test_interior_rhs_is_the_galerkin_integral():
    # b_p = int grad F_p . V, V = sum_o V_o F_o: Galerkin A a = b, so the
    # unit-free right-hand side of L27 chi = b27 is -b (h = 1)
    rng = np.random.default_rng(1)
    n = 7
    V = rng.standard_normal((n, n, n, 3))
    b27 = Q.divergence27(V, remove_mean=False)
    p = (3, 3, 3)
    for comp in range(3):
        Vc = np.zeros_like(V)
        Vc[..., comp] = V[..., comp]
        bc = Q.divergence27(Vc, remove_mean=False)[p]
        tot = 0.0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    def f(X, Y, Z):
                        g = [_hat(X), _hat(Y), _hat(Z)]
                        g[comp] = [_dhat(X), _dhat(Y), _dhat(Z)][comp]
                        return g[0] * g[1] * g[2] * _hat(X - dx) * _hat(Y - dy) * _hat(Z - dz)
                    tot += V[p[0] + dz, p[1] + dy, p[2] + dx, comp] * _cells_quadrature(f)
        assert abs(bc + tot) < 1e-12
    assert np.isfinite(b27).all()


def test_dct_modes_are_eigenvectors_with_the_closed_form():
    # the mirrored walls make the cosine modes exact eigenvectors, boundary rows included
    n = 10
    lam = Q.eigenvalues(n, n, n)
    for k in [(0, 0, 1), (3, 0, 0), (2, 5, 7), (9, 9, 9)]:
        v = P.dct_mode(n, k)
        Lv = Q.laplacian27(v)
        assert np.abs(Lv - lam[k[2], k[1], k[0]] * v).max() < 1e-12


def test_lumping_identity_gives_the_7_point_forms():
    # with M replaced by the identity the operator and divergence are the
    # transverse-lumped ones of poisson / divergence
    rng = np.random.default_rng(2)
    x = rng.standard_normal((6, 7, 8))
    s = sum(Q.stiffness_1d(x, a) for a in range(3))
    assert np.allclose(-s, P.laplacian(x), atol=1e-13)
    V = rng.standard_normal((6, 7, 8, 3))
    d = np.zeros(x.shape)
    for xi in range(3):
        Vxi = np.zeros_like(V)
        Vxi[..., xi] = V[..., xi]
        d += D.divergence(Vxi, remove_mean=False)
    assert np.allclose(d, D.divergence(V, remove_mean=False), atol=1e-13)


def test_symmetry_null_space_adjoint_and_solve():
    rng = np.random.default_rng(3)
    u = rng.standard_normal((6, 9, 8))
    v = rng.standard_normal((6, 9, 8))
    assert abs(np.sum(Q.laplacian27(u) * v) - np.sum(u * Q.laplacian27(v))) < 1e-10
    assert np.abs(Q.laplacian27(np.ones((6, 9, 8)))).max() < 1e-14
    # -L27 is positive semi-definite
    assert np.sum(-Q.laplacian27(u) * u) > 0
    V = rng.standard_normal((6, 9, 8, 3))
    g = rng.standard_normal((6, 9, 8))
    lhs = np.sum(Q.divergence27(V) * g)
    rhs = np.sum(V * Q.divergence27_adjoint(g))
    assert abs(lhs - rhs) < 1e-10
    assert abs(Q.divergence27(V).sum()) < 1e-10      # consistent Neumann system
    b = Q.divergence27(V)
    chi = Q.solve27(b)
    assert np.abs(Q.laplacian27(chi) - b).max() < 1e-11
    assert abs(chi.mean()) < 1e-13


def test_second_order_consistency():
    # L27 chi ~ h^2 Laplacian(chi) on a smooth field, error O(h^4)
    errs = []
    for n in (16, 32):
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        chi = np.cos(np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(np.pi * Z)
        lap = -(np.pi ** 2 + 4 * np.pi ** 2 + np.pi ** 2) * chi
        errs.append(np.abs(Q.laplacian27(chi) - h * h * lap).max() / (h * h))
    assert errs[1] < errs[0] / 3.5


def test_q1_chain_matches_central_fd():
    # the whole Q1 forward (splat, 27-point divergence and solve, iso-value,
    # marching cubes, exact distance) against its adjoint, bins frozen
    import synth
    from oracle import pipeline as PL
    res = 12
    p, n = synth.sphere_cloud(250, seed=7)
    p = p.astype(np.float64)
    n = n.astype(np.float64)
    bbox = np.array([0, 0, 0, 1, 1, 1], np.float32)
    rng = np.random.default_rng(4)
    g = rng.standard_normal((res, res, res))
    rec = PL.reconstruct(p, n, bbox, res, with_normals=False, operator="q1")
    dp, dn, _ = PL.backward(rec, g)

    def loss(pp, nn):
        r = PL.reconstruct(pp, nn, bbox, res, with_normals=False, frozen_bins=rec.bins, operator="q1")
        return float(np.sum(g * r.phi))

    eps = 1e-6
    for i, ax in [(2, 0), (40, 1), (111, 2)]:
        for arr, grad, is_p in ((p, dp, True), (n, dn, False)):
            a1, a2 = arr.copy(), arr.copy()
            a1[i, ax] += eps
            a2[i, ax] -= eps
            f1 = loss(a1, n) if is_p else loss(p, a1)
            f2 = loss(a2, n) if is_p else loss(p, a2)
            fd = (f1 - f2) / (2 * eps)
            assert abs(fd - grad[i, ax]) <= 1e-6 * max(1.0, abs(fd)) + 1e-6 * np.abs(grad).max()
    # the two operators give different but close surfaces on the same cloud
    lump = PL.reconstruct(p, n, bbox, res, with_normals=False)
    assert 0 < np.abs(lump.phi - rec.phi).max() < 0.5 / res
