"""torch.autograd wrapper: the forward runs wgeo_reconstruct + wgeo_query, the
backward runs wgeo_backward (adjoint chain with one transposed Poisson solve,
Sec. 2.5, Eqs. 35-39).  No solver iterate is saved; the handle keeps chi, c,
the bins, the triangles and the closest-triangle ids of the forward.  A
handle keeps only its last forward: each Function saves the forward's
generation number, and its backward raises StaleForwardError if the same
Reconstructor has run another forward since (rather than differentiate the
wrong state)."""
from __future__ import annotations

import torch

from .api import Reconstructor, sh_surface, sh_surface_backward


class WgeoQueryFunction(torch.autograd.Function):
    """(points, normals, q) -> (phi(q), n(q)) through a Reconstructor."""

    @staticmethod
    def forward(ctx, points, normals, q, recon: Reconstructor, bbox, res: int):
        recon.reconstruct(points.contiguous(), normals.contiguous(), bbox, res,
                          with_sdf=False, with_normals=False)
        sdf_q, nrm_q = recon.query(q.contiguous())
        ctx.recon = recon
        ctx.generation = recon.generation
        ctx.save_for_backward(q)
        return sdf_q, nrm_q

    @staticmethod
    def backward(ctx, g_sdf_q, g_nrm_q):
        (q,) = ctx.saved_tensors
        ctx.recon.check_generation(ctx.generation, "WgeoQueryFunction.backward")
        need_q = ctx.needs_input_grad[2]
        gs = g_sdf_q.contiguous() if g_sdf_q is not None else None
        gn = g_nrm_q.contiguous() if g_nrm_q is not None else None
        dp, dn, dq = ctx.recon.backward(q=q.contiguous(), d_sdf_q=gs, d_nrm_q=gn, want_dq=need_q)
        return dp, dn, dq, None, None, None


class WgeoExactQueryFunction(torch.autograd.Function):
    """(points, normals, q) -> exact phi(q) (off-grid distance to the
    reconstructed surface, Sec. 2.4) through a Reconstructor; the gradient of
    phi(q) is saved for d/dq and the mesh adjoint reruns the query search."""

    @staticmethod
    def forward(ctx, points, normals, q, recon: Reconstructor, bbox, res: int):
        recon.reconstruct(points.contiguous(), normals.contiguous(), bbox, res,
                          with_sdf=False, with_normals=False)
        sdf_q, _ = recon.query_exact(q.contiguous(), with_grad=False)
        ctx.recon = recon
        ctx.generation = recon.generation
        ctx.save_for_backward(q)
        return sdf_q

    @staticmethod
    def backward(ctx, g_sdf_q):
        (q,) = ctx.saved_tensors
        ctx.recon.check_generation(ctx.generation, "WgeoExactQueryFunction.backward")
        dp, dn, dq = ctx.recon.backward_exact(q.contiguous(), g_sdf_q.contiguous(),
                                              want_dq=ctx.needs_input_grad[2])
        return dp, dn, dq, None, None, None


class WgeoGridFunction(torch.autograd.Function):
    """(points, normals) -> (phi grid [res]^3, normal grid [3][res]^3)."""

    @staticmethod
    def forward(ctx, points, normals, recon: Reconstructor, bbox, res: int):
        sdf, nrm = recon.reconstruct(points.contiguous(), normals.contiguous(), bbox, res)
        ctx.recon = recon
        ctx.generation = recon.generation
        return sdf, nrm

    @staticmethod
    def backward(ctx, g_sdf, g_nrm):
        ctx.recon.check_generation(ctx.generation, "WgeoGridFunction.backward")
        dp, dn, _ = ctx.recon.backward(
            d_sdf_grid=g_sdf.contiguous() if g_sdf is not None else None,
            d_nrm_grid=g_nrm.contiguous() if g_nrm is not None else None)
        return dp, dn, None, None, None


class SHSurfaceFunction(torch.autograd.Function):
    """theta -> (points, normals) of the SH star body at fixed directions."""

    @staticmethod
    def forward(ctx, theta, dirs, recon: Reconstructor, base: float):
        pts, nrm = sh_surface(theta.contiguous(), dirs.contiguous(), base)
        ctx.save_for_backward(theta, dirs)
        ctx.recon = recon
        ctx.base = base
        return pts, nrm

    @staticmethod
    def backward(ctx, g_pts, g_nrm):
        theta, dirs = ctx.saved_tensors
        gp = g_pts.contiguous() if g_pts is not None else torch.zeros((dirs.shape[0], 3), device=dirs.device)
        gn = g_nrm.contiguous() if g_nrm is not None else torch.zeros((dirs.shape[0], 3), device=dirs.device)
        dth = sh_surface_backward(ctx.recon, theta.contiguous(), dirs, gp, gn, ctx.base)
        return dth, None, None, None


# The general entry: (points, normals, q) -> (phi(q), n(q)), differentiable in
# all three.
WgeoFunction = WgeoQueryFunction


def sdf_query(points, normals, q, recon: Reconstructor, bbox, res: int):
    return WgeoQueryFunction.apply(points, normals, q, recon, bbox, res)


def sdf_query_exact(points, normals, q, recon: Reconstructor, bbox, res: int):
    return WgeoExactQueryFunction.apply(points, normals, q, recon, bbox, res)


def sdf_grid(points, normals, recon: Reconstructor, bbox, res: int):
    return WgeoGridFunction.apply(points, normals, recon, bbox, res)


def sh_points(theta, dirs, recon: Reconstructor, base: float = 0.3):
    return SHSurfaceFunction.apply(theta, dirs, recon, base)
