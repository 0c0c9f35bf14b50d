"""Right-hand side b = <grad F_p, V> (Sec. 2.3, Eqs. 22 and 26).

With the trilinear basis of Eq. 16 and the two transverse axes integrated by
the nodal (trapezoid) rule, the one-dimensional integral int F'_p F_o is
{+1/2, 0, -1/2} for o = p-1, p, p+1, so b is a central divergence of the cell
coefficients V.  Written in conservative face form with zero flux through the
domain faces (the Neumann condition that the weak form of Eq. 19 implies):

    F_{xi, p+1/2} = (V_{p, xi} + V_{p+e_xi, xi}) / 2   on interior faces, 0 on domain faces
    b_p = sum_xi (F_{xi, p+1/2} - F_{xi, p-1/2})

(unit-free: the factors of h only rescale chi, and the SDF does not change
under chi -> s chi + t).  Finally the mean of b is removed so that the
singular Neumann system is consistent.
"""
from __future__ import annotations

import numpy as np

# numpy axis of each coordinate direction for [z, y, x] arrays
NP_AXIS = (2, 1, 0)


def _shift_faces(Vc: np.ndarray, ax: int) -> np.ndarray:
    """Face values along numpy axis ax: F[0..n] with F[0] = F[n] = 0."""
    n = Vc.shape[ax]
    shape = list(Vc.shape)
    shape[ax] = n + 1
    F = np.zeros(shape)
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    mid = [slice(None)] * 3
    lo[ax] = slice(0, n - 1)
    hi[ax] = slice(1, n)
    mid[ax] = slice(1, n)
    F[tuple(mid)] = 0.5 * (Vc[tuple(lo)] + Vc[tuple(hi)])
    return F


def divergence(V: np.ndarray, remove_mean: bool = True) -> np.ndarray:
    b = np.zeros(V.shape[:3])
    for xi in range(3):
        ax = NP_AXIS[xi]
        F = _shift_faces(V[..., xi], ax)
        n = V.shape[ax]
        up = [slice(None)] * 3
        dn = [slice(None)] * 3
        up[ax] = slice(1, n + 1)
        dn[ax] = slice(0, n)
        b += F[tuple(up)] - F[tuple(dn)]
    if remove_mean:
        b -= b.mean()
    return b


def divergence_adjoint(db: np.ndarray, remove_mean: bool = True) -> np.ndarray:
    """Transpose of ``divergence``: dL/dV [.., 3] from dL/db."""
    g = db - db.mean() if remove_mean else db
    dV = np.zeros(db.shape + (3,))
    for xi in range(3):
        ax = NP_AXIS[xi]
        n = db.shape[ax]
        # face p+1/2 (p = 0..n-2) contributes +g_p - g_{p+1}; it takes
        # (V_p + V_{p+1}) / 2, so both cells receive half of that.
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        face = 0.5 * (g[tuple(lo)] - g[tuple(hi)])
        dV[tuple(lo) + (xi,)] += face
        dV[tuple(hi) + (xi,)] += face
    return dV
