"""Poisson solve A a = b (Sec. 2.3, Eqs. 15, 20, 21) on the uniform grid.

With the transverse-lumped trilinear basis, A_{p,o} = <grad F_p, grad F_o> is
the cell-centred 7-point operator with zero-flux (Neumann) domain faces.  The
oracle uses the unit-free graph Laplacian

    (L chi)_p = sum_{q in-grid neighbour of p} (chi_q - chi_p)

(L = -A up to a factor h) and solves L chi = b with the gauge sum(chi) = 0.

The solve is exact (to FP64 rounding) and direct: the DCT-II basis
v_k(i) = prod_xi cos(pi k_xi (i_xi + 1/2) / n) diagonalises L with eigenvalue
lambda_k = -4 sum_xi sin^2(pi k_xi / (2 n)); the k = 0 mode (the constant
null space) is dropped.  A plain FP64 conjugate-gradient solve is kept as an
independent cross-check.
"""
from __future__ import annotations

import numpy as np


def laplacian(chi: np.ndarray) -> np.ndarray:
    out = np.zeros_like(chi, dtype=np.float64)
    for ax in range(3):
        n = chi.shape[ax]
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        d = chi[tuple(hi)] - chi[tuple(lo)]          # chi_{p+1} - chi_p across each interior face
        out[tuple(lo)] += d
        out[tuple(hi)] -= d
    return out


def dct_matrix(n: int) -> np.ndarray:
    """Orthonormal DCT-II matrix Q[k, i] = s_k cos(pi k (i + 1/2) / n)."""
    k = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    Q = np.cos(np.pi * k * (i + 0.5) / n)
    Q[0] *= np.sqrt(1.0 / n)
    Q[1:] *= np.sqrt(2.0 / n)
    return Q


def eigenvalues_1d(n: int) -> np.ndarray:
    return -4.0 * np.sin(np.pi * np.arange(n) / (2.0 * n)) ** 2


def _apply_axis(Q: np.ndarray, x: np.ndarray, ax: int) -> np.ndarray:
    y = np.tensordot(Q, x, axes=([1], [ax]))       # new axis 0
    return np.moveaxis(y, 0, ax)


def solve(b: np.ndarray) -> np.ndarray:
    """chi with L chi = b - mean(b) and sum(chi) = 0."""
    nz, ny, nx = b.shape
    Qs = [dct_matrix(nz), dct_matrix(ny), dct_matrix(nx)]
    bh = b - b.mean()
    for ax in range(3):
        bh = _apply_axis(Qs[ax], bh, ax)
        # bh <- Q along ax (forward transform)
    lam = (eigenvalues_1d(nz)[:, None, None] + eigenvalues_1d(ny)[None, :, None]
           + eigenvalues_1d(nx)[None, None, :])
    lam[0, 0, 0] = 1.0
    ch = bh / lam
    ch[0, 0, 0] = 0.0
    for ax in range(3):
        ch = _apply_axis(Qs[ax].T, ch, ax)
    return ch


def dct_mode(n: int, k) -> np.ndarray:
    """Unnormalised eigenvector cos(pi k_x (i+1/2)/n) cos(..y..) cos(..z..), [z,y,x]."""
    i = np.arange(n) + 0.5
    cx = np.cos(np.pi * k[0] * i / n)
    cy = np.cos(np.pi * k[1] * i / n)
    cz = np.cos(np.pi * k[2] * i / n)
    return cz[:, None, None] * cy[None, :, None] * cx[None, None, :]


def mode_eigenvalue(n: int, k) -> float:
    return float(sum(-4.0 * np.sin(np.pi * kk / (2.0 * n)) ** 2 for kk in k))


def cg(b: np.ndarray, tol: float = 1e-13, maxiter: int = 10000) -> np.ndarray:
    """Plain conjugate gradients on -L (SPD on mean-zero vectors)."""
    rhs = -(b - b.mean())
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    nb = np.sqrt(float(np.sum(rhs * rhs)))
    if nb == 0:
        return x
    for _ in range(maxiter):
        Ap = -laplacian(p)
        alpha = rr / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.sum(r * r))
        if np.sqrt(rr_new) <= tol * nb:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x - x.mean()
