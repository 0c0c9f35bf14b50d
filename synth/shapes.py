"""Seeded synthetic shapes standing in for the paper's point clouds.

The paper's fish / aircraft / car / jet / vascular clouds (Sec. 3.1) are not
available, so every workload is an analytic body sampled with a fixed seed:

* sphere: centre (0.5, 0.5, 0.5), radius 0.3, points uniform on the surface
  (normalised Gaussian directions), exact outward normals;
* star bodies r(u) = 0.3 + sum_k theta_k Y_k(u) with orthonormal real spherical
  harmonics Y_k (no Condon-Shortley phase, index k = l*l + l + m), sampled
  either area-uniformly (rejection on the surface Jacobian) or at fixed seeded
  directions (differentiable in theta);
* an ellipsoid (semi-axes 0.35/0.08/0.12) bent by a lateral travelling wave
  0.04 s^2 sin(2 pi (s/0.9 - t/T)), s = (x - x_head)/L, L = 0.7, T = 200 steps.

Normals of a star body come from the implicit form F(x) = |x - c| - r(u):
grad F = u - P_perp grad r / r, where P_perp projects on the tangent plane.
Spherical harmonics are evaluated in Cartesian form (a polynomial in z times
Re/Im (x + i y)^m), so there is no pole singularity.
"""
from __future__ import annotations

import functools
import math

import numpy as np

CENTRE = np.array([0.5, 0.5, 0.5])
# seed per workload: 1000 + index of the workload in the list
#   0 sphere 64^3, 1 SH body 256^3, 2 differentiable SH body 128^3,
#   3 moving ellipsoid 192^3, 4 serving mix
CONFIG_SEEDS = {"sphere64": 1000, "shbody256": 1001, "shopt128": 1002,
                "wave192": 1003, "serving": 1004}


def sh_count(lmax: int) -> int:
    return (lmax + 1) ** 2


def real_sh(lmax: int, dirs: np.ndarray, grad: bool = False):
    """Orthonormal real SH up to degree lmax at unit directions dirs [n,3].

    Returns Y [n, K] and, if grad, the Cartesian gradient of the polynomial
    extension dY [n, K, 3] (project it on the tangent plane for the surface
    gradient).
    """
    d = np.asarray(dirs, dtype=np.float64)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    n = d.shape[0]
    K = sh_count(lmax)
    Y = np.zeros((n, K))
    dY = np.zeros((n, K, 3)) if grad else None
    # C_m + i S_m = (x + i y)^m
    C = [np.ones(n)]
    S = [np.zeros(n)]
    for m in range(1, lmax + 1):
        C.append(x * C[m - 1] - y * S[m - 1])
        S.append(x * S[m - 1] + y * C[m - 1])
    for m in range(0, lmax + 1):
        # Q_l^m(z): P_l^m(z) = (1 - z^2)^{m/2} Q_l^m(z), positive convention
        dfact = 1.0
        for j in range(1, 2 * m, 2):
            dfact *= j
        Q = {m: np.full(n, dfact)}
        dQ = {m: np.zeros(n)}
        if m + 1 <= lmax:
            Q[m + 1] = (2 * m + 1) * z * Q[m]
            dQ[m + 1] = (2 * m + 1) * (Q[m] + z * dQ[m])
        for l in range(m + 2, lmax + 1):
            Q[l] = ((2 * l - 1) * z * Q[l - 1] - (l + m - 1) * Q[l - 2]) / (l - m)
            dQ[l] = ((2 * l - 1) * (Q[l - 1] + z * dQ[l - 1])
                     - (l + m - 1) * dQ[l - 2]) / (l - m)
        for l in range(m, lmax + 1):
            Klm = math.sqrt((2 * l + 1) / (4 * math.pi)
                            * math.factorial(l - m) / math.factorial(l + m))
            if m == 0:
                k = l * l + l
                Y[:, k] = Klm * Q[l]
                if grad:
                    dY[:, k, 2] = Klm * dQ[l]
            else:
                s2 = math.sqrt(2.0) * Klm
                kc = l * l + l + m
                ks = l * l + l - m
                Y[:, kc] = s2 * Q[l] * C[m]
                Y[:, ks] = s2 * Q[l] * S[m]
                if grad:
                    dY[:, kc, 0] = s2 * Q[l] * m * C[m - 1]
                    dY[:, kc, 1] = s2 * Q[l] * (-m) * S[m - 1]
                    dY[:, kc, 2] = s2 * dQ[l] * C[m]
                    dY[:, ks, 0] = s2 * Q[l] * m * S[m - 1]
                    dY[:, ks, 1] = s2 * Q[l] * m * C[m - 1]
                    dY[:, ks, 2] = s2 * dQ[l] * S[m]
    return (Y, dY) if grad else Y


def _lmax_of(theta: np.ndarray) -> int:
    l = int(round(math.sqrt(len(theta)))) - 1
    assert (l + 1) ** 2 == len(theta), "theta length must be (lmax+1)^2"
    return l


def sh_surface(theta: np.ndarray, dirs: np.ndarray, base: float = 0.3,
               centre: np.ndarray = CENTRE):
    """Points and outward unit normals of r(u) = base + sum theta_k Y_k(u)."""
    theta = np.asarray(theta, dtype=np.float64)
    u = np.asarray(dirs, dtype=np.float64)
    Y, dY = real_sh(_lmax_of(theta), u, grad=True)
    r = base + Y @ theta
    g = np.einsum("nkc,k->nc", dY, theta)
    g = g - np.sum(g * u, axis=1, keepdims=True) * u          # tangential part
    m = u - g / r[:, None]
    nrm = m / np.linalg.norm(m, axis=1, keepdims=True)
    pts = centre[None, :] + r[:, None] * u
    return pts, nrm, r


def sh_surface_vjp(theta: np.ndarray, dirs: np.ndarray, dpts: np.ndarray,
                   dnrm: np.ndarray, base: float = 0.3) -> np.ndarray:
    """d/dtheta of sum(dpts * pts) + sum(dnrm * nrm) for sh_surface (fixed dirs)."""
    theta = np.asarray(theta, dtype=np.float64)
    u = np.asarray(dirs, dtype=np.float64)
    dpts = np.asarray(dpts, dtype=np.float64)
    dnrm = np.asarray(dnrm, dtype=np.float64)
    Y, dY = real_sh(_lmax_of(theta), u, grad=True)
    G = dY - np.einsum("nkc,nc->nk", dY, u)[:, :, None] * u[:, None, :]  # tangential
    r = base + Y @ theta
    g = np.einsum("nkc,k->nc", G, theta)
    m = u - g / r[:, None]
    mn = np.linalg.norm(m, axis=1, keepdims=True)
    n = m / mn
    dm = (dnrm - np.sum(dnrm * n, axis=1, keepdims=True) * n) / mn
    # x = c + r u           -> dx/dtheta_k = Y_k u
    out = np.einsum("nk,n->k", Y, np.sum(dpts * u, axis=1))
    # m = u - g / r          -> dm/dtheta_k = -G_k / r + g Y_k / r^2
    out += -np.einsum("nkc,nc->k", G, dm / r[:, None])
    out += np.einsum("nk,n->k", Y, np.sum(dm * g, axis=1) / r ** 2)
    return out


def uniform_dirs(n: int, rng: np.random.Generator) -> np.ndarray:
    g = rng.standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


@functools.lru_cache(maxsize=8)
def _grid_sh(lmax: int, grid: tuple):
    """Real SH up to lmax on a (theta, phi) grid of directions."""
    th = np.linspace(0.0, math.pi, grid[0])
    ph = np.linspace(0.0, 2 * math.pi, grid[1], endpoint=False)
    T, P = np.meshgrid(th, ph, indexing="ij")
    u = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    return real_sh(lmax, u)


def _fit_perturbation(theta: np.ndarray, base: float, rmax: float = 0.45,
                      rmin: float = 0.1, grid=(256, 512)):
    """Scale the perturbation so base + perturbation stays in [rmin, rmax]
    (checked on a (theta, phi) grid of the given size)."""
    pert = _grid_sh(_lmax_of(theta), tuple(grid)) @ theta
    s = 1.0
    if pert.max() > rmax - base:
        s = min(s, (rmax - base) / pert.max())
    if pert.min() < rmin - base:
        s = min(s, (rmin - base) / pert.min())
    return theta * s, s


def sphere_cloud(n: int = 4096, seed: int = CONFIG_SEEDS["sphere64"],
                 radius: float = 0.3, centre=CENTRE):
    rng = np.random.default_rng(seed)
    u = uniform_dirs(n, rng)
    pts = np.asarray(centre)[None, :] + radius * u
    return pts.astype(np.float32), u.astype(np.float32)


def random_sh_theta(lmax: int, rng: np.random.Generator, std: float = 0.02):
    return rng.normal(0.0, std, sh_count(lmax))


def random_sh_body_theta(lmax: int, rng: np.random.Generator, std: float = 0.02, base: float = 0.3,
                         grid=(64, 128)):
    """Coefficients of a random SH star body (N(0, std^2)), the perturbation
    scaled into [0.1, 0.45] on a coarse direction grid (one body per request
    of the serving mix)."""
    theta, _ = _fit_perturbation(random_sh_theta(lmax, rng, std), base, grid=grid)
    return theta


def sh_body_cloud(n: int = 200_000, lmax: int = 8, seed: int = CONFIG_SEEDS["shbody256"],
                  noise: float = 0.002, std: float = 0.02, base: float = 0.3):
    """Area-uniform samples of a random SH star body, analytic normals, then
    Gaussian position noise.  Returns (points f32, normals f32, info dict)."""
    rng = np.random.default_rng(seed)
    theta, scale = _fit_perturbation(random_sh_theta(lmax, rng, std), base)

    def jac(u):
        Y, dY = real_sh(lmax, u, grad=True)
        r = base + Y @ theta
        g = np.einsum("nkc,k->nc", dY, theta)
        g = g - np.sum(g * u, axis=1, keepdims=True) * u
        return r * np.sqrt(r * r + np.sum(g * g, axis=1))

    jmax = 1.25 * jac(uniform_dirs(20000, np.random.default_rng(seed + 7))).max()
    keep = []
    got = 0
    while got < n:
        u = uniform_dirs(max(2 * (n - got), 1024), rng)
        acc = rng.random(len(u)) * jmax < jac(u)
        keep.append(u[acc])
        got += int(acc.sum())
    u = np.concatenate(keep)[:n]
    pts, nrm, _ = sh_surface(theta, u, base)
    if noise > 0:
        pts = pts + rng.normal(0.0, noise, pts.shape)
    return pts.astype(np.float32), nrm.astype(np.float32), {"theta": theta, "scale": scale}


def sh_fixed_dirs_cloud(n: int = 100_000, lmax: int = 6, seed: int = CONFIG_SEEDS["shopt128"],
                        std: float = 0.02, base: float = 0.3):
    """Fixed seeded directions and two coefficient vectors (start, target) of
    the differentiable SH body.  Returns (dirs f64, theta0 f64, theta_target f64)."""
    rng = np.random.default_rng(seed)
    dirs = uniform_dirs(n, rng)
    th0, _ = _fit_perturbation(random_sh_theta(lmax, rng, std), base)
    tht, _ = _fit_perturbation(random_sh_theta(lmax, rng, std), base)
    return dirs, th0.astype(np.float32).astype(np.float64), tht.astype(np.float32).astype(np.float64)


def wave_ellipsoid_cloud(t: int, n: int = 50_000, seed: int = CONFIG_SEEDS["wave192"],
                         axes=(0.35, 0.08, 0.12), amp: float = 0.04, wavelength: float = 0.9,
                         period: int = 200):
    """Ellipsoid bent by a travelling lateral wave, resampled at step t."""
    a = np.asarray(axes, dtype=np.float64)
    rng = np.random.default_rng(seed + t)
    L = 2 * a[0]
    x_head = CENTRE[0] - a[0]

    def area_factor(u):
        return np.linalg.norm(u / a[None, :], axis=1)

    fmax = 1.0 / a.min()
    keep, got = [], 0
    while got < n:
        u = uniform_dirs(2 * (n - got) + 1024, rng)
        acc = rng.random(len(u)) * fmax < area_factor(u)
        keep.append(u[acc])
        got += int(acc.sum())
    u = np.concatenate(keep)[:n]
    p = CENTRE[None, :] + u * a[None, :]
    nrm = u / a[None, :]
    s = (p[:, 0] - x_head) / L
    ph = 2 * math.pi * (s / wavelength - t / period)
    g = amp * s * s * np.sin(ph)
    gx = (2 * amp * s * np.sin(ph) + amp * s * s * np.cos(ph) * 2 * math.pi / wavelength) / L
    p[:, 1] += g
    nn = np.stack([nrm[:, 0] - gx * nrm[:, 1], nrm[:, 1], nrm[:, 2]], axis=1)
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    return p.astype(np.float32), nn.astype(np.float32)


def uniform_queries(m: int, seed: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return (lo + rng.random((m, 3)) * (hi - lo)).astype(np.float32)


def serving_requests(count: int = 2000, seed: int = CONFIG_SEEDS["serving"]):
    """The serving mix: per request grid size, point count, gradient flag and a
    unit-rate exponential inter-arrival gap (scale it by 1/rate)."""
    rng = np.random.default_rng(seed)
    res = rng.choice([64, 128, 256], size=count, p=[0.5, 0.35, 0.15])
    npts = np.exp(rng.uniform(math.log(10_000), math.log(500_000), count)).astype(np.int64)
    grad = rng.random(count) < 0.5
    gaps = rng.exponential(1.0, count)
    return [{"id": i, "res": int(res[i]), "n": int(npts[i]), "grad": bool(grad[i]),
             "gap": float(gaps[i]), "seed": 50_000 + i} for i in range(count)]


def config_inputs(name: str, small: bool = False):
    """Inputs of a named workload: dict(points, normals, bbox, res, queries, ...)."""
    bbox = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
    if name == "sphere64":
        p, n = sphere_cloud()
        return dict(points=p, normals=n, bbox=bbox, res=64,
                    queries=uniform_queries(100_000, 2000))
    if name == "shbody256":
        p, n, info = sh_body_cloud()
        return dict(points=p, normals=n, bbox=bbox, res=256,
                    queries=uniform_queries(1_000_000, 2001), info=info)
    if name == "shopt128":
        dirs, th0, tht = sh_fixed_dirs_cloud()
        p, n, _ = sh_surface(th0, dirs)
        return dict(points=p.astype(np.float32), normals=n.astype(np.float32), bbox=bbox,
                    res=128, queries=uniform_queries(500_000, 2002), dirs=dirs,
                    theta=th0, theta_target=tht)
    if name == "wave192":
        p, n = wave_ellipsoid_cloud(0)
        return dict(points=p, normals=n, bbox=bbox, res=192,
                    queries=uniform_queries(100_000, 2003))
    raise KeyError(name)
