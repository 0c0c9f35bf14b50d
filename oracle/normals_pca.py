"""Distance-weighted PCA normal estimation (Sec. 2.1, the four displayed
equations of the neighbourhood, the weights, the weighted centroid and
Eq. weighted_covariance, then the eigen-decomposition).  Test infrastructure
only: the CUDA path never imports it.

For every point x_i:
  N_i   = { x_j : |x_j - x_i| <= R }          (x_i itself included)
  w_ij  = 1 / (|x_j - x_i| + eps)
  xbar  = sum_j w_ij x_j / W_i,   W_i = sum_j w_ij
  C_i   = sum_j w_ij (x_j - xbar)(x_j - xbar)^T / W_i
  n_i   = eigenvector of C_i with the smallest eigenvalue (unit, unoriented)

A neighbourhood of fewer than 3 points, or a covariance with no positive
eigenvalue, has no normal: the zero vector is returned.  The sign of n_i is
not part of the definition; callers compare directions up to sign.

Membership |x_j - x_i| <= R decides an integer (who is a neighbour), so it is
taken in the paper's precision, float32 (its kernels run in Warp's float32):
the differences, their squares and the two sums each rounded to float32, in
the order ((dx^2 + dy^2) + dz^2), against R^2 rounded to float32.  Everything
after the membership (weights, centroid, covariance, eigenvectors) is FP64.
`exact_ball=True` takes the FP64 test instead (the mathematical ball).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def dpca_point(x, neighbours, eps):
    """Normal, ascending eigenvalues and neighbour count of one point from its
    neighbourhood (an array that includes x itself)."""
    X = np.asarray(neighbours, dtype=np.float64)
    if len(X) < 3:
        return np.zeros(3), np.zeros(3), len(X)
    d = np.linalg.norm(X - x, axis=1)
    w = 1.0 / (d + eps)
    W = w.sum()
    xbar = (w[:, None] * X).sum(axis=0) / W
    Y = X - xbar
    C = (w[:, None, None] * (Y[:, :, None] * Y[:, None, :])).sum(axis=0) / W
    lam, V = np.linalg.eigh(C)
    if not lam[-1] > 0.0:
        return np.zeros(3), lam, len(X)
    return V[:, 0], lam, len(X)


def in_ball_f32(P32, i, cand, radius: float):
    """The members of `cand` (indices) within `radius` of point i, decided in
    float32 as described in the module docstring."""
    cand = np.asarray(cand, dtype=np.int64)
    d = P32[cand] - P32[i]
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    r = np.float32(radius)
    return cand[d2 <= r * r]


def _finite(P):
    return np.isfinite(P).all(axis=1)


def dpca_normals(points, radius: float, eps: float, exact_ball: bool = False):
    """(normals [n,3], eigenvalues [n,3] ascending, neighbour counts [n]) for all
    points; neighbourhoods from a k-d tree ball query.  Points with a non-finite
    coordinate take part in no neighbourhood and get the zero normal."""
    P = np.asarray(points, dtype=np.float64)
    n = len(P)
    normals = np.zeros((n, 3))
    lam = np.zeros((n, 3))
    cnt = np.zeros(n, dtype=np.int64)
    ok = _finite(P) if n else np.zeros(0, dtype=bool)
    if not ok.any():
        return normals, lam, cnt
    idx = np.nonzero(ok)[0]
    Q = P[idx]
    Q32 = Q.astype(np.float32)
    tree = cKDTree(Q)
    # float32 membership can admit a point a few float32 ulps beyond R: query a
    # slightly larger ball and let the float32 test decide
    nbrs = tree.query_ball_point(Q, radius if exact_ball else radius * (1 + 1e-5))
    for k, i in enumerate(idx):
        nb = np.asarray(nbrs[k], dtype=np.int64) if exact_ball else in_ball_f32(Q32, k, nbrs[k], radius)
        normals[i], lam[i], cnt[i] = dpca_point(P[i], Q[nb], eps)
    return normals, lam, cnt


def dpca_normals_brute(points, radius: float, eps: float, exact_ball: bool = False):
    """The same by testing every pair (small clouds)."""
    P = np.asarray(points, dtype=np.float64)
    n = len(P)
    normals = np.zeros((n, 3))
    lam = np.zeros((n, 3))
    cnt = np.zeros(n, dtype=np.int64)
    ok = _finite(P) if n else np.zeros(0, dtype=bool)
    idx = np.nonzero(ok)[0]
    Q = P[idx]
    Q32 = Q.astype(np.float32)
    for k, i in enumerate(idx):
        if exact_ball:
            nb = np.nonzero(np.linalg.norm(Q - Q[k], axis=1) <= radius)[0]
        else:
            nb = in_ball_f32(Q32, k, np.arange(len(Q)), radius)
        normals[i], lam[i], cnt[i] = dpca_point(P[i], Q[nb], eps)
    return normals, lam, cnt
