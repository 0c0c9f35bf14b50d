"""Surface normals from the SDF gradient, n = grad phi / |grad phi| (Sec. 2.4,
the unit-normal statement after Eq. 32).

grad_h phi uses central differences (phi_{p+1} - phi_{p-1}) / (2h) inside and
the second-order one-sided forms (-3 phi_0 + 4 phi_1 - phi_2) / (2h) and
(3 phi_{n-1} - 4 phi_{n-2} + phi_{n-3}) / (2h) on the first and last node of an
axis.  n = 0 where |grad_h phi| = 0 or where the gradient is not finite.
Output layout: [3, z, y, x] (one plane per component).
"""
from __future__ import annotations

import numpy as np

from .divergence import NP_AXIS


def grad_axis(phi, ax, h):
    n = phi.shape[ax]
    g = np.zeros_like(phi)

    def s(i):
        sl = [slice(None)] * 3
        sl[ax] = i
        return tuple(sl)

    g[s(slice(1, n - 1))] = (phi[s(slice(2, n))] - phi[s(slice(0, n - 2))]) / (2 * h)
    g[s(0)] = (-3 * phi[s(0)] + 4 * phi[s(1)] - phi[s(2)]) / (2 * h)
    g[s(n - 1)] = (3 * phi[s(n - 1)] - 4 * phi[s(n - 2)] + phi[s(n - 3)]) / (2 * h)
    return g


def gradient(phi, h):
    return np.stack([grad_axis(phi, NP_AXIS[xi], h) for xi in range(3)], axis=0)


def normals(phi, h):
    g = gradient(phi, h)
    with np.errstate(invalid="ignore", divide="ignore"):
        mag = np.sqrt(np.sum(g * g, axis=0))
        ok = np.isfinite(mag) & (mag > 0)
        n = np.where(ok[None], g / np.where(ok, mag, 1.0)[None], 0.0)
    return n, g, mag


def grad_axis_adjoint(dg, ax, h):
    """Transpose of grad_axis."""
    n = dg.shape[ax]
    out = np.zeros_like(dg)

    def s(i):
        sl = [slice(None)] * 3
        sl[ax] = i
        return tuple(sl)

    inner = dg[s(slice(1, n - 1))] / (2 * h)
    out[s(slice(2, n))] += inner
    out[s(slice(0, n - 2))] -= inner
    g0 = dg[s(0)] / (2 * h)
    out[s(0)] += -3 * g0
    out[s(1)] += 4 * g0
    out[s(2)] += -g0
    gl = dg[s(n - 1)] / (2 * h)
    out[s(n - 1)] += 3 * gl
    out[s(n - 2)] += -4 * gl
    out[s(n - 3)] += gl
    return out


def normals_adjoint(phi, h, dn):
    """dL/dphi from dL/dn [3, z, y, x]."""
    n, g, mag = normals(phi, h)
    ok = np.isfinite(mag) & (mag > 0)
    proj = dn - n * np.sum(n * dn, axis=0, keepdims=True)
    dg = np.where(ok[None], proj / np.where(ok, mag, 1.0)[None], 0.0)
    out = np.zeros_like(phi)
    for xi in range(3):
        out += grad_axis_adjoint(dg[xi], NP_AXIS[xi], h)
    return out
