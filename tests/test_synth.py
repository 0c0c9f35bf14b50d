"""Pins for the seeded input generators (not the method): real SH
orthonormality, star-body normals, and the differentiable generator's VJP."""
import math

import numpy as np
import pytest

import synth
from synth.shapes import real_sh, sh_surface, sh_surface_vjp


def _sphere_quadrature(nt=40, nph=80):
    x, w = np.polynomial.legendre.leggauss(nt)
    ph = np.arange(nph) * 2 * math.pi / nph
    Z, P = np.meshgrid(x, ph, indexing="ij")
    W = np.meshgrid(w, ph, indexing="ij")[0] * 2 * math.pi / nph
    s = np.sqrt(1 - Z ** 2)
    u = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    return u, W.reshape(-1)


def test_real_sh_orthonormal():
    u, w = _sphere_quadrature()
    Y = real_sh(8, u)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(81)).max() < 1e-12


def test_real_sh_low_degree_closed_forms():
    u = synth.uniform_dirs(50, np.random.default_rng(0))
    Y = real_sh(1, u)
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[:, 0], c0)
    assert np.allclose(Y[:, 1], c1 * u[:, 1])     # l=1, m=-1 ~ y
    assert np.allclose(Y[:, 2], c1 * u[:, 2])     # m=0 ~ z
    assert np.allclose(Y[:, 3], c1 * u[:, 0])     # m=1 ~ x


def test_star_body_normals_are_surface_normals():
    rng = np.random.default_rng(1)
    theta = rng.normal(0, 0.02, 49)
    u = synth.uniform_dirs(40, rng)
    pts, nrm, r = sh_surface(theta, u)
    # tangent vectors by finite differences along two directions on the sphere
    for i in range(len(u)):
        t1 = np.cross(u[i], [0.3, 0.5, 0.8])
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(u[i], t1)
        for t in (t1, t2):
            e = 1e-6
            up = (u[i] + e * t)
            um = (u[i] - e * t)
            up /= np.linalg.norm(up)
            um /= np.linalg.norm(um)
            pp, _, _ = sh_surface(theta, up[None])
            pm, _, _ = sh_surface(theta, um[None])
            tang = (pp[0] - pm[0]) / (2 * e)
            assert abs(np.dot(tang, nrm[i])) < 1e-6 * np.linalg.norm(tang)
        assert np.dot(nrm[i], u[i]) > 0


def test_generator_vjp_fd():
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 0.02, 49)
    u = synth.uniform_dirs(30, rng)
    dp = rng.standard_normal((30, 3))
    dn = rng.standard_normal((30, 3))
    g = sh_surface_vjp(theta, u, dp, dn)
    for k in (0, 5, 17, 48):
        e = 1e-7
        tp = theta.copy()
        tm = theta.copy()
        tp[k] += e
        tm[k] -= e
        fp = np.sum(sh_surface(tp, u)[0] * dp) + np.sum(sh_surface(tp, u)[1] * dn)
        fm = np.sum(sh_surface(tm, u)[0] * dp) + np.sum(sh_surface(tm, u)[1] * dn)
        assert (fp - fm) / (2 * e) == pytest.approx(g[k], rel=1e-6, abs=1e-8)


def test_seeded_and_shapes():
    p1, n1 = synth.sphere_cloud(100)
    p2, n2 = synth.sphere_cloud(100)
    assert np.array_equal(p1, p2) and p1.dtype == np.float32
    assert np.allclose(np.linalg.norm(p1 - 0.5, axis=1), 0.3, atol=1e-6)
    p, n, info = synth.sh_body_cloud(2000)
    r = np.linalg.norm(p - 0.5, axis=1)
    assert r.min() > 0.08 and r.max() < 0.47
    pw, nw = synth.wave_ellipsoid_cloud(10, n=1000)
    assert pw.shape == (1000, 3) and np.allclose(np.linalg.norm(nw, axis=1), 1, atol=1e-6)
    reqs = synth.serving_requests(200)
    assert {r["res"] for r in reqs} <= {64, 128, 256}
    assert all(10_000 <= r["n"] <= 500_000 for r in reqs)
