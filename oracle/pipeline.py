"""The whole path, forward and adjoint, in FP64 (Sec. 2.3-2.5).

reconstruct:  points, normals -> bins -> V (Eqs. 23-25) -> b (Eqs. 22, 26)
              -> chi (Eqs. 20-21) -> c (Eq. 27) -> triangles (Eq. 28)
              -> phi = sign * min distance (Eqs. 29-34) -> n = grad phi / |grad phi|
query:        trilinear phi and normalised trilinear n at query points
backward:     the adjoint chain (Eqs. 35-39).  The stiffness matrix does not
              depend on the points (Eq. 21; the box and grid are inputs), so
              dA/dtheta = 0 and Eq. 39 reduces to lambda^T db/dtheta with
              A^T lambda = dL/da (Eq. 38); the Laplacian is symmetric, so the
              adjoint solve is the forward solve.  Discrete choices (central
              cell, marching-cubes case, closest triangle and feature) are held
              fixed: the derivative of the piecewise-smooth branch.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import divergence as D
from . import galerkin_q1 as Q1
from . import grid as G
from . import iso as I
from . import mc as M
from . import normals as NR
from . import poisson as P
from . import sdf as S
from . import splat as SP


@dataclass
class Reconstruction:
    res: int
    h: float
    lo: np.ndarray
    points: np.ndarray
    normals_in: np.ndarray
    bins: np.ndarray
    finite: np.ndarray
    status: int
    V: np.ndarray
    b: np.ndarray
    chi: np.ndarray
    c: float
    mesh: dict
    phi: np.ndarray | None = None          # [z,y,x] (full grid only)
    dist: np.ndarray | None = None
    tri: np.ndarray | None = None
    sign: np.ndarray | None = None
    nrm: np.ndarray | None = None          # [3,z,y,x]
    gmag: np.ndarray | None = None
    extra: dict = field(default_factory=dict)
    operator: str = "lumped"               # "lumped": 7-point forms; "q1": unlumped Galerkin


def as_f64(a):
    """float32 inputs are promoted; float64 inputs (finite-difference checks) are kept."""
    a = np.asarray(a)
    if a.dtype == np.float64:
        return a
    return a.astype(np.float32).astype(np.float64)


def forward_to_mesh(points, normals, bbox, res, frozen_bins=None, operator: str = "lumped"):
    """Stages up to and including marching cubes.

    ``frozen_bins`` replaces the central cells (used by finite-difference
    checks, so that both sides differentiate the same smooth branch).
    ``operator``: "lumped" (the 7-point operator and face divergence) or "q1"
    (the unlumped trilinear Galerkin forms of `galerkin_q1`)."""
    lo = G.grid_lo(bbox)
    h = G.grid_spacing(bbox, res)
    p = as_f64(points)
    nr = as_f64(normals)
    bins, finite, status = G.bin_points(p, bbox, res)
    if frozen_bins is not None:
        bins = np.asarray(frozen_bins, dtype=np.int64)
    V = SP.splat(p, nr, bins, finite, lo, h, res)
    if operator == "q1":
        b = Q1.divergence27(V)
        chi = Q1.solve27(b)
    elif operator == "lumped":
        b = D.divergence(V)
        chi = P.solve(b)
    else:
        raise ValueError(operator)
    c = I.isovalue(chi, p, finite, lo, h, res)
    mesh = M.marching_cubes(chi, c, lo, h)
    if mesh["gid"].shape[0] == 0:
        status |= G.STATUS_EMPTY_SURFACE
    return Reconstruction(res=res, h=h, lo=lo, points=p, normals_in=nr, bins=bins,
                          finite=finite, status=status, V=V, b=b, chi=chi, c=c, mesh=mesh,
                          operator=operator)


def node_xyz(lin, res, lo, h):
    z, rem = np.divmod(np.asarray(lin, dtype=np.int64), res * res)
    y, x = np.divmod(rem, res)
    return lo[None, :] + (np.stack([x, y, z], axis=1) + 0.5) * h


def sdf_at(rec: Reconstruction, lin):
    """phi, distance and closest triangle at the given linear node indices."""
    nodes = node_xyz(lin, rec.res, rec.lo, rec.h)
    chi_flat = rec.chi.reshape(-1)
    sgn = S.node_sign(chi_flat[lin], rec.c)
    if rec.mesh["verts"].shape[0] == 0:
        return sgn * np.inf, np.full(len(lin), np.inf), np.full(len(lin), -1)
    d, tri = S.exact_distance(nodes, rec.mesh["verts"])
    return sgn * d, d, tri


def sdf_at_pool(rec: Reconstruction, lin, workers: int = 1, pool=None):
    """sdf_at, with the exact distance evaluated by `workers` processes (or by
    an existing process pool)."""
    nodes = node_xyz(lin, rec.res, rec.lo, rec.h)
    sgn = S.node_sign(rec.chi.reshape(-1)[lin], rec.c)
    if rec.mesh["verts"].shape[0] == 0:
        return sgn * np.inf, np.full(len(lin), np.inf), np.full(len(lin), -1)
    d, tri = S.exact_distance_pool(nodes, rec.mesh["verts"], workers, pool=pool)
    return sgn * d, d, tri


def fill_nodes(rec: Reconstruction, lin, workers: int = 1):
    """Evaluates phi, the distance and the closest triangle of a forward
    (`forward_to_mesh`) at the linear node indices `lin` only (NaN / -1 at
    every other node, no normals).  Enough for `backward` with grid or query
    seeds of phi whose nodes (query corners included) all lie in `lin`; every
    value it holds is the one `reconstruct` computes."""
    res = rec.res
    lin = np.unique(np.asarray(lin, dtype=np.int64))
    N = res ** 3
    phi = np.full(N, np.nan)
    dist = np.full(N, np.nan)
    tri = np.full(N, -1, dtype=np.int64)
    phi[lin], dist[lin], tri[lin] = sdf_at_pool(rec, lin, workers)
    rec.phi = phi.reshape(res, res, res)
    rec.dist = dist.reshape(res, res, res)
    rec.tri = tri.reshape(res, res, res)
    rec.sign = S.node_sign(rec.chi, rec.c)
    return rec


def reconstruct_at_nodes(points, normals, bbox, res, lin, workers: int = 1, frozen_bins=None):
    """`forward_to_mesh`, then `fill_nodes` at the linear node indices `lin`."""
    return fill_nodes(forward_to_mesh(points, normals, bbox, res, frozen_bins), lin, workers)


def query_corner_nodes(q, res, lo, h):
    """Linear indices of the 8 trilinear corner nodes of every query point."""
    corners, _, _ = I.trilinear(as_f64(q), lo, h, res)
    return np.unique(((corners[..., 2] * res + corners[..., 1]) * res + corners[..., 0]).reshape(-1))


def reconstruct(points, normals, bbox, res, with_normals: bool = True, frozen_bins=None,
                operator: str = "lumped", workers: int = 1):
    """The whole forward on the full grid (`workers` > 1: the exact distance
    evaluated by a process pool, `sdf_at_pool`)."""
    rec = forward_to_mesh(points, normals, bbox, res, frozen_bins, operator)
    N = res ** 3
    phi, d, tri = sdf_at_pool(rec, np.arange(N), workers)
    rec.phi = phi.reshape(res, res, res)
    rec.dist = d.reshape(res, res, res)
    rec.tri = tri.reshape(res, res, res)
    rec.sign = S.node_sign(rec.chi, rec.c)
    if with_normals:
        if np.isfinite(rec.phi).all():
            rec.nrm, _, rec.gmag = NR.normals(rec.phi, rec.h)
        else:
            rec.nrm = np.zeros((3, res, res, res))
            rec.gmag = np.zeros((res, res, res))
    return rec


def normals_at(rec: Reconstruction, lin):
    """Stencil normals at the given nodes, computing phi only where needed."""
    res = rec.res
    z, rem = np.divmod(np.asarray(lin, dtype=np.int64), res * res)
    y, x = np.divmod(rem, res)
    idx = np.stack([x, y, z], axis=1)
    need = {}
    taps = []
    for ax in range(3):
        i = idx[:, ax]
        lo_side = i == 0
        hi_side = i == res - 1
        offs_c = [(-1, -0.5), (1, 0.5)]
        tl = []
        for k in range(len(i)):
            if lo_side[k]:
                tl.append([(0, -1.5), (1, 2.0), (2, -0.5)])
            elif hi_side[k]:
                tl.append([(0, 1.5), (-1, -2.0), (-2, 0.5)])
            else:
                tl.append(offs_c)
        taps.append(tl)
    allnodes = []
    for k in range(len(idx)):
        for ax in range(3):
            for off, _w in taps[ax][k]:
                q = idx[k].copy()
                q[ax] += off
                allnodes.append((q[2] * res + q[1]) * res + q[0])
    uniq = np.unique(np.array(allnodes, dtype=np.int64))
    phi_u, _, _ = sdf_at(rec, uniq)
    lookup = dict(zip(uniq.tolist(), phi_u.tolist()))
    g = np.zeros((len(idx), 3))
    for k in range(len(idx)):
        for ax in range(3):
            acc = 0.0
            for off, w in taps[ax][k]:
                q = idx[k].copy()
                q[ax] += off
                acc += w * lookup[int((q[2] * res + q[1]) * res + q[0])]
            g[k, ax] = acc / rec.h
    mag = np.linalg.norm(g, axis=1)
    ok = np.isfinite(mag) & (mag > 0)
    n = np.where(ok[:, None], g / np.where(ok, mag, 1.0)[:, None], 0.0)
    return n, mag


def query(rec: Reconstruction, q):
    qq = as_f64(q)
    sdf_q = I.interpolate(rec.phi, qq, rec.lo, rec.h, rec.res)
    nn = np.moveaxis(rec.nrm, 0, -1)                       # [z,y,x,3]
    m = I.interpolate(nn, qq, rec.lo, rec.h, rec.res)
    mag = np.linalg.norm(m, axis=1)
    nrm_q = np.where(mag[:, None] > 0, m / np.where(mag > 0, mag, 1.0)[:, None], 0.0)
    return sdf_q, nrm_q


def backward(rec: Reconstruction, d_sdf_grid=None, d_nrm_grid=None, q=None,
             d_sdf_q=None, d_nrm_q=None, return_parts: bool = False, q_exact=None, d_sdf_exact=None):
    """(d_points [n,3], d_normals [n,3], d_q [m,3] or None).

    q_exact / d_sdf_exact: seeds dL/dphi(q) of the exact off-grid distance
    (Eqs. 30 and 33 at arbitrary q, `query_exact`).  They enter like the
    node seeds, through the closest point of each query's closest triangle:
    d phi / d y = -s u, u = (q - y) / |q - y|.  With them, the returned d_q is
    that of the exact queries (s u times the seed)."""
    res, h, lo = rec.res, rec.h, rec.lo
    dphi = np.zeros((res, res, res))
    dn = np.zeros((3, res, res, res))
    if d_sdf_grid is not None:
        dphi += np.asarray(d_sdf_grid, dtype=np.float64).reshape(res, res, res)
    if d_nrm_grid is not None:
        dn += np.asarray(d_nrm_grid, dtype=np.float64).reshape(3, res, res, res)
    dq = None
    if q is not None:
        qq = as_f64(q)
        corners, w, dw = I.trilinear(qq, lo, h, res)
        dq = np.zeros_like(qq)
        if d_sdf_q is not None:
            g = np.asarray(d_sdf_q, dtype=np.float64)
            np.add.at(dphi, (corners[..., 2], corners[..., 1], corners[..., 0]), w * g[:, None])
            phic = I.gather(rec.phi, corners)
            dq += np.einsum("nc,ncx->nx", phic * g[:, None], dw)
        if d_nrm_q is not None:
            gq = np.asarray(d_nrm_q, dtype=np.float64)
            nn = np.moveaxis(rec.nrm, 0, -1)
            nc = I.gather(nn, corners)                        # [m,8,3]
            m = np.einsum("nc,nck->nk", w, nc)
            mag = np.linalg.norm(m, axis=1)
            ok = mag > 0
            nq = np.where(ok[:, None], m / np.where(ok, mag, 1.0)[:, None], 0.0)
            dm = np.where(ok[:, None], (gq - nq * np.sum(nq * gq, 1, keepdims=True))
                          / np.where(ok, mag, 1.0)[:, None], 0.0)
            for k in range(3):
                np.add.at(dn[k], (corners[..., 2], corners[..., 1], corners[..., 0]),
                          w * dm[:, k:k + 1])
            dq += np.einsum("nck,nk,ncx->nx", nc, dm, dw)
    # normals stencil adjoint
    if np.any(dn != 0):
        dphi += NR.normals_adjoint(rec.phi, h, dn)
    # SDF adjoint: phi_o = s_o |p_o - y_o|, y_o = sum_v beta_v P_v
    verts = rec.mesh["verts"]
    T = verts.shape[0]
    dP = np.zeros((T, 3, 3))
    if q_exact is not None and d_sdf_exact is not None and T > 0:
        from . import query_exact as QE
        qe = as_f64(q_exact)
        ge = np.asarray(d_sdf_exact, dtype=np.float64)
        phi_e, grad_e, tri_e = QE.query_exact(qe, verts)
        act_e = (ge != 0) & (tri_e >= 0)
        y, bary = S.closest_point_triangle(qe[act_e], verts[tri_e[act_e], 0], verts[tri_e[act_e], 1],
                                           verts[tri_e[act_e], 2])
        coef = -ge[act_e, None] * grad_e[act_e]                        # -s u dL/dphi
        for v in range(3):
            np.add.at(dP[:, v, :], tri_e[act_e], bary[:, v:v + 1] * coef)
        dq = grad_e * ge[:, None]
    flat = dphi.reshape(-1)
    act = np.nonzero(flat)[0]
    if T > 0 and len(act):
        tri = rec.tri.reshape(-1)[act]
        nodes = node_xyz(act, res, lo, h)
        y, bary = S.closest_point_triangle(nodes, verts[tri, 0], verts[tri, 1], verts[tri, 2])
        diff = nodes - y
        d = np.linalg.norm(diff, axis=1)
        ok = d > 0
        u = np.where(ok[:, None], diff / np.where(ok, d, 1.0)[:, None], 0.0)
        sgn = rec.sign.reshape(-1)[act]
        coef = -(sgn * flat[act])[:, None] * u                         # d phi / d y
        for v in range(3):
            np.add.at(dP[:, v, :], tri, bary[:, v:v + 1] * coef)
    # marching-cubes adjoint: vertex = lower node + eta h e_axis
    dchi = np.zeros((res, res, res))
    dc = 0.0
    if T > 0:
        gid = rec.mesh["gid"]
        eta, c1, c2, p, axis = M.edge_eta(rec.chi, rec.c, gid)
        deta = h * np.take_along_axis(dP, axis[..., None], axis=2)[..., 0]   # [T,3]
        den = c2 - c1
        g1 = deta * (eta - 1.0) / den
        g2 = -deta * eta / den
        dc = float(np.sum(deta / den))
        q2 = p.copy()
        for a in range(3):
            q2[..., a] += (axis == a)
        np.add.at(dchi, (p[..., 2], p[..., 1], p[..., 0]), g1)
        np.add.at(dchi, (q2[..., 2], q2[..., 1], q2[..., 0]), g2)
    # iso-value adjoint: c = mean_i chi_hat(x_i)
    dpts_iso = np.zeros_like(rec.points)
    fin = rec.finite
    npf = int(fin.sum())
    if npf > 0 and dc != 0.0:
        corners, w, dw = I.trilinear(rec.points[fin], lo, h, res)
        np.add.at(dchi, (corners[..., 2], corners[..., 1], corners[..., 0]), w * (dc / npf))
        chic = I.gather(rec.chi, corners)
        dpts_iso[fin] = np.einsum("nc,ncx->nx", chic, dw) * (dc / npf)
    # adjoint solve (L symmetric): lambda = L^+ P dchi
    if rec.operator == "q1":
        lam = Q1.solve27(dchi)
        dV = Q1.divergence27_adjoint(lam)
    else:
        lam = P.solve(dchi)
        dV = D.divergence_adjoint(lam)
    dpts, dnrm = SP.splat_adjoint(rec.points, rec.normals_in, rec.bins, rec.finite, lo, h, res, dV)
    dpts = dpts + dpts_iso
    if return_parts:
        return dpts, dnrm, dq, {"dphi": dphi, "dP": dP, "dchi": dchi, "dc": dc,
                                "lam": lam, "dV": dV, "dpts_iso": dpts_iso}
    return dpts, dnrm, dq
