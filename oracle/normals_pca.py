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


def dpca_normals(points, radius: float, eps: float):
    """(normals [n,3], eigenvalues [n,3] ascending, neighbour counts [n]) for all
    points; neighbourhoods from a k-d tree ball query."""
    P = np.asarray(points, dtype=np.float64)
    n = len(P)
    normals = np.zeros((n, 3))
    lam = np.zeros((n, 3))
    cnt = np.zeros(n, dtype=np.int64)
    if n == 0:
        return normals, lam, cnt
    tree = cKDTree(P)
    nbrs = tree.query_ball_point(P, radius)
    for i in range(n):
        normals[i], lam[i], cnt[i] = dpca_point(P[i], P[nbrs[i]], eps)
    return normals, lam, cnt


def dpca_normals_brute(points, radius: float, eps: float):
    """The same by testing every pair (small clouds)."""
    P = np.asarray(points, dtype=np.float64)
    n = len(P)
    normals = np.zeros((n, 3))
    lam = np.zeros((n, 3))
    cnt = np.zeros(n, dtype=np.int64)
    for i in range(n):
        d = np.linalg.norm(P - P[i], axis=1)
        normals[i], lam[i], cnt[i] = dpca_point(P[i], P[d <= radius], eps)
    return normals, lam, cnt
