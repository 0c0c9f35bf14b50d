"""Shape-parameter gradient of the differentiable workload, in FP64
(Sec. 2.5, last paragraph, and Sec. 3.3; reading R11 for the loss).

A star body with spherical-harmonic radius r(u; theta) is sampled at fixed
unit directions u_i (the input generator ``synth.sh_surface``); its points
and normals are reconstructed (Sec. 2.3-2.4) and the loss is the mean
squared mismatch of the interpolated signed distance at fixed query points
against a target's:

    L(theta) = (1/M) sum_j (phi(q_j; theta) - phi_target(q_j))^2.

dL/dtheta is the adjoint of the whole chain: the query seeds
2 (phi - phi_target) / M go through ``pipeline.backward`` (Eqs. 35-39) to the
points and normals, and from there through the generator's vector-Jacobian
product ``synth.sh_surface_vjp``.  phi is evaluated only at the query corners
(``pipeline.reconstruct_at_nodes``), which is all the loss and its adjoint
read.
"""
from __future__ import annotations

import numpy as np

from . import iso as I
from . import pipeline as P


def sh_cloud(theta, dirs, float32: bool = True):
    """Points and normals of the body (float32-rounded, as a GPU caller holds
    them, or FP64 for finite differences)."""
    from synth.shapes import sh_surface
    p, n, _ = sh_surface(np.asarray(theta, dtype=np.float64), np.asarray(dirs, dtype=np.float64))
    if float32:
        return p.astype(np.float32), n.astype(np.float32)
    return p, n


def phi_at_queries(points, normals, q, bbox, res, workers: int = 1, frozen_bins=None):
    """(phi(q) [M], the reconstruction) with phi at the query corners only."""
    rec0 = P.forward_to_mesh(points, normals, bbox, res, frozen_bins)
    lin = P.query_corner_nodes(q, res, rec0.lo, rec0.h)
    rec = P.reconstruct_at_nodes(points, normals, bbox, res, lin, workers, frozen_bins)
    return I.interpolate(rec.phi, P.as_f64(q), rec.lo, rec.h, res), rec


def loss(phi_q, phi_target):
    d = np.asarray(phi_q, dtype=np.float64) - np.asarray(phi_target, dtype=np.float64)
    return float(np.mean(d * d))


def loss_seeds(phi_q, phi_target):
    """dL/dphi(q_j) = 2 (phi(q_j) - phi_target(q_j)) / M."""
    d = np.asarray(phi_q, dtype=np.float64) - np.asarray(phi_target, dtype=np.float64)
    return 2.0 * d / len(d)


def theta_gradient(theta, dirs, rec, q, seeds):
    """dL/dtheta = VJP of the generator applied to the adjoint chain's
    (dL/dpoints, dL/dnormals); also returns those two."""
    from synth.shapes import sh_surface_vjp
    dp, dn, _ = P.backward(rec, q=q, d_sdf_q=seeds)
    dth = sh_surface_vjp(np.asarray(theta, dtype=np.float64), np.asarray(dirs, dtype=np.float64), dp, dn)
    return dth, dp, dn
