"""Unlumped trilinear Galerkin operator and right-hand side (Sec. 2.3,
Eqs. 15-22 and 26, with F of Eq. 16 the trilinear hat, not lumped).  Test
infrastructure only: the CUDA path never imports it.

With F(t) = max(0, 1 - |t|) per axis at the cell centres, the Galerkin
integrals factor into one-dimensional ones:

    int F'_p F'_o = {-1, 2, -1} / h     (stiffness S)
    int F_p F_o   = h {1/6, 2/3, 1/6}   (mass M = I - S/6)
    int F'_p F_o  = {+1/2, 0, -1/2}     (o = p-1, p, p+1)

so A = S (x) M (x) M + M (x) S (x) M + M (x) M (x) S, a 27-point stencil
(interior: centre 8/3, faces 0, edges -1/6, corners -1/12, times h), and
b_p = <grad F_p, V> = sum_xi (D_xi (x) M (x) M) V_xi with D the central
difference.  The domain faces: the basis is mirrored at the walls (the
homogeneous Neumann condition of the weak form): the coefficient of the
mirror cell of a cell outside the grid is that of the cell inside, and the
normal component of V flips sign there, so D is the face-form difference
with zero flux through the walls (as in `divergence`), and S, M take the
rows S_00 = 1, M_00 = 5/6 at the ends.  Replacing M by the identity gives
the transverse-lumped operator and divergence of `poisson` and `divergence`.

Unit-free forms (the h factors only rescale chi, see `divergence`):

    (L27 chi) = -(S M M + M S M + M M S) chi     (the sign of `poisson.laplacian`)
    b27       = sum_xi M_eta M_zeta (D_xi V_xi), mean removed

Both one-dimensional factors are diagonalised by the DCT-II basis (S with
eigenvalues 4 sin^2(pi k / 2n), M with 1 - that / 6), so the solve is a
direct DCT solve like `poisson.solve`.
"""
from __future__ import annotations

import numpy as np

from . import divergence as D
from . import poisson as P

NP_AXIS = D.NP_AXIS


def _mirror_neighbours(x: np.ndarray, ax: int):
    """(x_{i-1}, x_{i+1}) along numpy axis ax with the walls mirrored."""
    n = x.shape[ax]
    idx_m = np.clip(np.arange(n) - 1, 0, n - 1)
    idx_p = np.clip(np.arange(n) + 1, 0, n - 1)
    return np.take(x, idx_m, axis=ax), np.take(x, idx_p, axis=ax)


def mass_1d(x: np.ndarray, ax: int) -> np.ndarray:
    """M along numpy axis ax: (2/3) x_i + (1/6)(x_{i-1} + x_{i+1}), mirrored."""
    xm, xp = _mirror_neighbours(x, ax)
    return (2.0 / 3.0) * x + (xm + xp) / 6.0


def stiffness_1d(x: np.ndarray, ax: int) -> np.ndarray:
    """S along numpy axis ax: 2 x_i - x_{i-1} - x_{i+1}, mirrored."""
    xm, xp = _mirror_neighbours(x, ax)
    return 2.0 * x - xm - xp


def laplacian27(chi: np.ndarray) -> np.ndarray:
    """-(S M M + M S M + M M S) chi."""
    chi = np.asarray(chi, dtype=np.float64)
    out = np.zeros_like(chi)
    for a in range(3):
        t = stiffness_1d(chi, a)
        for b in range(3):
            if b != a:
                t = mass_1d(t, b)
        out -= t
    return out


def divergence27(V: np.ndarray, remove_mean: bool = True) -> np.ndarray:
    """sum_xi M M (D_xi V_xi), D the face-form difference of `divergence`."""
    b = np.zeros(V.shape[:3])
    for xi in range(3):
        Vxi = np.zeros_like(V)
        Vxi[..., xi] = V[..., xi]
        t = D.divergence(Vxi, remove_mean=False)
        for b_ax in range(3):
            if b_ax != NP_AXIS[xi]:
                t = mass_1d(t, b_ax)
        b += t
    if remove_mean:
        b -= b.mean()
    return b


def divergence27_adjoint(db: np.ndarray, remove_mean: bool = True) -> np.ndarray:
    """Transpose of ``divergence27``: dL/dV [.., 3] from dL/db (M is symmetric)."""
    g = db - db.mean() if remove_mean else np.asarray(db, dtype=np.float64)
    dV = np.zeros(g.shape + (3,))
    for xi in range(3):
        t = g
        for b_ax in range(3):
            if b_ax != NP_AXIS[xi]:
                t = mass_1d(t, b_ax)
        dV[..., xi] = D.divergence_adjoint(t, remove_mean=False)[..., xi]
    return dV


def eigenvalues(nz: int, ny: int, nx: int) -> np.ndarray:
    """Eigenvalues of L27 on the DCT-II modes [kz, ky, kx]."""
    lz, ly, lx = (4.0 * np.sin(np.pi * np.arange(n) / (2.0 * n)) ** 2 for n in (nz, ny, nx))
    mz, my, mx = 1.0 - lz / 6.0, 1.0 - ly / 6.0, 1.0 - lx / 6.0
    return -(lz[:, None, None] * my[None, :, None] * mx[None, None, :]
             + mz[:, None, None] * ly[None, :, None] * mx[None, None, :]
             + mz[:, None, None] * my[None, :, None] * lx[None, None, :])


def solve27(b: np.ndarray) -> np.ndarray:
    """chi with L27 chi = b - mean(b) and sum(chi) = 0 (direct DCT solve)."""
    nz, ny, nx = b.shape
    Qs = [P.dct_matrix(nz), P.dct_matrix(ny), P.dct_matrix(nx)]
    bh = b - b.mean()
    for ax in range(3):
        bh = P._apply_axis(Qs[ax], bh, ax)
    lam = eigenvalues(nz, ny, nx)
    lam[0, 0, 0] = 1.0
    ch = bh / lam
    ch[0, 0, 0] = 0.0
    for ax in range(3):
        ch = P._apply_axis(Qs[ax].T, ch, ax)
    return ch
