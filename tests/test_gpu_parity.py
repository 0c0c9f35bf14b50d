"""GPU path vs the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerances (stated by the method's target): bins bit-exact; SDF max |diff| <=
1e-4 of the box extent; normals within 0.1 degree (nodes where the oracle's
|grad_h phi| < 0.9 — medial axis — excluded); gradients within 1e-4 relative
(L2) of the oracle's adjoint, and every point's gradient within 1e-4 of the
largest one.  Sizes span several 8^3 splat tiles and 4^3 marching-cubes
bricks and end in ragged partial tiles.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import grid as OG
from oracle import pipeline as OP

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BBOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
SDF_TOL = 1e-4          # 1e-4 of the unit box extent
ANGLE_TOL_DEG = 0.1
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_2609_20964_gb300 import Reconstructor
    torch.cuda.set_device(0)
    return Reconstructor


def _cases():
    out = {}
    p, n = synth.sphere_cloud(1500, seed=21)
    out["sphere24"] = (p, n, 24)
    p, n, _ = synth.sh_body_cloud(6000, seed=22, noise=0.002)
    out["shbody44"] = (p, n, 44)
    p, n = synth.wave_ellipsoid_cloud(37, n=5000)
    out["wave40"] = (p, n, 40)
    return out


CASES = _cases()
_ORACLE = {}


def _oracle(name):
    if name not in _ORACLE:
        p, n, res = CASES[name]
        _ORACLE[name] = oracle.reconstruct(p, n, BBOX, res)
    return _ORACLE[name]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _smooth_nodes(ref):
    """Nodes whose gradient stencil (+-2 along each axis) stays off the medial
    axis (oracle |grad_h phi| >= 0.9): there the normal and its adjoint are
    defined and the closest triangles are not near-ties."""
    bad = ref.gmag < 0.9
    near = bad.copy()
    for ax in range(3):
        for s in (1, -1, 2, -2):
            near |= np.roll(bad, s, axis=ax)
    return ~near


def _check_grad(got, want, nm):
    """Relative 2-norm error <= GRAD_TOL, and every point's error <= GRAD_TOL
    of the largest per-point gradient (a cluster of wrong points cannot hide
    in the norm)."""
    got = got.cpu().numpy().astype(np.float64) if hasattr(got, "cpu") else np.asarray(got, np.float64)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= GRAD_TOL, f"{nm}: relative error {rel:.3e}"
    pp = np.linalg.norm((got - want).reshape(len(want), -1), axis=1).max()
    scale = np.linalg.norm(np.asarray(want).reshape(len(want), -1), axis=1).max()
    assert pp <= GRAD_TOL * scale, f"{nm}: largest per-point error {pp / scale:.3e} of the largest gradient"


def _angle_deg(a, b):
    # float64 and atan2(|a x b|, a . b): arccos of a float32-normalised dot
    # product near 1 would itself carry ~0.02 degrees of rounding
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.degrees(np.arctan2(cr, np.sum(a * b, axis=-1)))


@pytest.mark.parametrize("name", list(CASES))
def test_forward_parity(W, name):
    p, n, res = CASES[name]
    ref = _oracle(name)
    rec = W(res, len(p))
    sdf, nrm = rec.reconstruct(_t(p), _t(n), BBOX, res)
    bins = rec.bins().cpu().numpy()
    b = rec.field("b").cpu().numpy().astype(np.float64)
    chi = rec.field("chi").cpu().numpy().astype(np.float64)
    info = rec.info()
    assert info["status"] == 0, info
    # S1: bins bit-exact
    assert np.array_equal(bins, ref.bins.astype(np.int32))
    # S3-S4: right-hand side to float32 rounding
    assert np.abs(b - ref.b).max() <= 2e-6 * np.abs(ref.b).max() + 1e-7
    # S5: chi up to the additive constant
    span = ref.chi.max() - ref.chi.min()
    assert np.abs((chi - chi.mean()) - (ref.chi - ref.chi.mean())).max() <= 1e-4 * span
    # S6: iso-value, relative to the spread of chi
    assert abs((info["isovalue"] - chi.mean()) - (ref.c - ref.chi.mean())) <= 1e-4 * span
    # S7-S8: signed distance
    phi = sdf.cpu().numpy().astype(np.float64)
    assert np.abs(phi - ref.phi).max() <= SDF_TOL
    # S9: normals away from the medial axis
    g = nrm.cpu().numpy().astype(np.float64)
    ok = ref.gmag >= 0.9
    ang = _angle_deg(np.moveaxis(g, 0, -1)[ok], np.moveaxis(ref.nrm, 0, -1)[ok])
    assert ang.max() <= ANGLE_TOL_DEG, f"max angle {ang.max()} deg"
    assert ok.mean() > 0.8
    rec.close()


@pytest.mark.parametrize("scale", [1.0, 37.0])
def test_splat_dense_and_sparse_tiles(W, scale):
    # a sparse sphere plus a dense cap: tiles with short point lists sum in two
    # 32-bit words, the dense ones (lists flushed) in 64-bit words; with
    # normals scaled by 37 the two-word rule admits lists of at most 824
    # points.  b must match the oracle either way (the integer sums are exact)
    rng = np.random.default_rng(31)
    p0, n0 = synth.sphere_cloud(400, seed=32)
    d = rng.standard_normal((6000, 3))
    d[:, 2] = np.abs(d[:, 2]) * 20.0          # directions near the +z pole
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p1 = (0.5 + 0.3 * d).astype(np.float32)
    p = np.concatenate([p0, p1]).astype(np.float32)
    n = (np.concatenate([n0, d.astype(np.float32)]) * scale).astype(np.float32)
    res = 40
    ref = OP.forward_to_mesh(p, n, BBOX, res)
    rec = W(res, len(p))
    rec.reconstruct(_t(p), _t(n), BBOX, res)
    b = rec.field("b").cpu().numpy().astype(np.float64)
    assert rec.info()["status"] == 0
    assert np.abs(b - ref.b).max() <= 2e-6 * np.abs(ref.b).max() + 1e-7
    # the dense cap does put more points in one tile than one list holds
    tiles = (np.asarray(rec.bins().cpu().numpy()) // 8)
    _, counts = np.unique(tiles, axis=0, return_counts=True)
    assert counts.max() > 3584
    rec.close()


@pytest.mark.parametrize("name", list(CASES))
def test_query_and_backward_parity(W, name):
    p, n, res = CASES[name]
    ref = _oracle(name)
    rng = np.random.default_rng(5)
    q = synth.uniform_queries(3000, seed=31)
    gs = rng.standard_normal(len(q)).astype(np.float32)
    gn = rng.standard_normal((len(q), 3)).astype(np.float32)
    rec = W(res, len(p))
    rec.reconstruct(_t(p), _t(n), BBOX, res)
    Q = _t(q)
    sq, nq = rec.query(Q)
    rs, rn = OP.query(ref, q)
    assert np.abs(sq.cpu().numpy() - rs).max() <= SDF_TOL
    # normals at queries whose 8 corner nodes are all off the medial axis
    from oracle import iso as OI
    corners, _, _ = OI.trilinear(q.astype(np.float64), ref.lo, ref.h, res)
    good = np.all(OI.gather(ref.gmag, corners) >= 0.9, axis=1)
    ang = _angle_deg(nq.cpu().numpy()[good], rn[good])
    good = np.all(OI.gather(_smooth_nodes(ref), corners), axis=1)
    assert ang.max() <= ANGLE_TOL_DEG
    # backward through the query loss (phi and normals at q) to points, normals and
    # q, seeded only at queries whose stencils stay off the medial axis: there phi
    # is not differentiable (two distinct closest points) and dn/dphi ~ 1/|grad phi|
    gn[~good] = 0.0
    gs[~good] = 0.0
    dp, dn, dq = rec.backward(q=Q, d_sdf_q=_t(gs), d_nrm_q=_t(gn), want_dq=True)
    odp, odn, odq = OP.backward(ref, q=q, d_sdf_q=gs.astype(np.float64), d_nrm_q=gn.astype(np.float64))
    for got, want, nm in ((dp, odp, "d_points"), (dn, odn, "d_normals"), (dq, odq, "d_q")):
        _check_grad(got, want, nm)
    rec.close()


@pytest.mark.parametrize("name", list(CASES))
def test_unmasked_phi_seed_backward_parity(W, name):
    """Seeds of phi at every query, medial axis included: nodes whose closest
    surface point jumps there are decided on the refined surface as the
    oracle decides them, so no seed needs masking."""
    p, n, res = CASES[name]
    ref = _oracle(name)
    q = synth.uniform_queries(4000, seed=33)
    gs = np.random.default_rng(6).standard_normal(len(q)).astype(np.float32)
    rec = W(res, len(p))
    rec.reconstruct(_t(p), _t(n), BBOX, res)
    Q = _t(q)
    dp, dn, dq = rec.backward(q=Q, d_sdf_q=_t(gs), want_dq=True)
    odp, odn, odq = OP.backward(ref, q=q, d_sdf_q=gs.astype(np.float64))
    for got, want, nm in ((dp, odp, "d_points"), (dn, odn, "d_normals"), (dq, odq, "d_q")):
        _check_grad(got, want, nm)
    rec.close()


@pytest.mark.parametrize("name", ["sphere24", "shbody44"])
def test_closest_point_parity(W, name):
    """S7 argmin: the closest surface point of every node, wherever the oracle
    finds it unique (no other triangle within 2e-7 of the minimum distance with
    a closest point more than 1e-6 away); triangle ids differ between the two
    meshes' orders, so the points are compared."""
    from oracle import sdf as S
    p, n, res = CASES[name]
    ref = _oracle(name)
    rec = W(res, len(p))
    rec.reconstruct(_t(p), _t(n), BBOX, res)
    ids = rec.field("closest").cpu().numpy().reshape(-1).astype(np.int64)
    vg, _ = rec.mesh()
    vg = vg.astype(np.float64)
    nodes = OP.node_xyz(np.arange(res ** 3), res, ref.lo, ref.h)
    vo = ref.mesh["verts"]
    to = ref.tri.reshape(-1)
    assert ids.min() >= 0 and ids.max() < len(vg)
    yg, _ = S.closest_point_triangle(nodes, vg[ids, 0], vg[ids, 1], vg[ids, 2])
    yo, _ = S.closest_point_triangle(nodes, vo[to, 0], vo[to, 1], vo[to, 2])
    amb = S.closest_point_ambiguous(nodes, vo, np.abs(ref.phi).reshape(-1), 2e-7, 1e-6)
    assert amb.mean() < 0.1, amb.mean()
    err = np.linalg.norm(yg - yo, axis=1)[~amb]
    assert err.max() <= 1e-5, f"closest point off by {err.max():.3e}"
    rec.close()


@pytest.mark.parametrize("res", [9, 12, 18, 28, 36, 40, 56])
def test_hierarchy_shapes_converge(W, res):
    """Grids whose multigrid hierarchies end differently (coarsest sizes 9, 6,
    9, 7, 9, 5, 7; zero to three levels above the one-CTA solve): the solve
    converges and the SDF matches the oracle."""
    p, n = synth.sphere_cloud(2000, seed=24)
    ref = oracle.reconstruct(p, n, BBOX, res)
    rec = W(res, len(p))
    sdf, _ = rec.reconstruct(_t(p), _t(n), BBOX, res)
    info = rec.info()
    assert info["status"] == 0, info
    assert np.abs(sdf.cpu().numpy().astype(np.float64) - ref.phi).max() <= SDF_TOL
    rec.close()


def test_odd_resolution(W):
    """An odd grid (15^3: no multigrid level above the one-CTA solve, pairs of
    cells ending in a single cell) against the oracle, forward and backward."""
    p, n = synth.sphere_cloud(1200, seed=23)
    res = 15
    ref = oracle.reconstruct(p, n, BBOX, res)
    rec = W(res, len(p))
    sdf, _ = rec.reconstruct(_t(p), _t(n), BBOX, res)
    assert rec.info()["status"] == 0
    assert np.abs(sdf.cpu().numpy().astype(np.float64) - ref.phi).max() <= SDF_TOL
    rng = np.random.default_rng(4)
    wg = rng.standard_normal((res, res, res)).astype(np.float32)
    wg[~_smooth_nodes(ref)] = 0.0
    dp, dn, _ = rec.backward(d_sdf_grid=_t(wg))
    odp, odn, _ = OP.backward(ref, d_sdf_grid=wg.astype(np.float64))
    for got, want, nm in ((dp, odp, "d_points"), (dn, odn, "d_normals")):
        _check_grad(got, want, nm)
    rec.close()


def test_grid_seed_backward_parity(W):
    p, n, res = CASES["sphere24"]
    ref = _oracle("sphere24")
    rng = np.random.default_rng(9)
    wg = rng.standard_normal((res, res, res)).astype(np.float32)
    wn = rng.standard_normal((3, res, res, res)).astype(np.float32)
    # normal seeds only where the normal is well defined (see _smooth_nodes)
    wn[:, ~_smooth_nodes(ref)] = 0.0
    wg[~_smooth_nodes(ref)] = 0.0
    rec = W(res, len(p))
    rec.reconstruct(_t(p), _t(n), BBOX, res)
    dp, dn, _ = rec.backward(d_sdf_grid=_t(wg), d_nrm_grid=_t(wn))
    odp, odn, _ = OP.backward(ref, d_sdf_grid=wg.astype(np.float64), d_nrm_grid=wn.astype(np.float64))
    for got, want, nm in ((dp, odp, "d_points"), (dn, odn, "d_normals")):
        _check_grad(got, want, nm)
    rec.close()


def test_deterministic_and_handle_reuse(W):
    p, n, res = CASES["shbody44"]
    rec = W(64, 20000)
    s1, n1 = rec.reconstruct(_t(p), _t(n), BBOX, res)
    s1 = s1.clone()
    n1 = n1.clone()
    # a different res on the same handle, then back
    p2, n2 = synth.sphere_cloud(3000, seed=3)
    rec.reconstruct(_t(p2), _t(n2), BBOX, 32)
    s2, n2b = rec.reconstruct(_t(p), _t(n), BBOX, res)
    assert torch.equal(s1, s2) and torch.equal(n1, n2b)
    rec.close()


@pytest.mark.parametrize("precision", ["mixed", "fp32"])
def test_graph_loop_equals_fixed_sequence(W, precision):
    """The solve recorded as a graph with a device-side loop and the same
    kernels enqueued as a fixed gated sequence give identical results,
    forward and backward."""
    from paper_2609_20964_gb300 import PREC_FP32, PREC_MIXED
    p, n, res = CASES["shbody44"]
    prec = PREC_FP32 if precision == "fp32" else PREC_MIXED
    q = _t(synth.uniform_queries(500, seed=7))
    g = _t(np.random.default_rng(8).standard_normal(500).astype(np.float32))
    out = []
    for use_graphs in (1, 0):
        rec = W(res, len(p), precision=prec, use_graphs=use_graphs, max_vcycles=60)
        sdf, nrm = rec.reconstruct(_t(p), _t(n), BBOX, res)
        sdf, nrm = sdf.clone(), nrm.clone()
        info = rec.info()
        dp = dn = None
        if precision == "mixed":
            dp, dn, _ = rec.backward(q=q, d_sdf_q=g)
            dp, dn = dp.clone(), dn.clone()
            info = rec.info()
        out.append((sdf, nrm, dp, dn, info["solver_steps"], info["backward_steps"], info["residual_rel"]))
        rec.close()
    a, b = out
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    if precision == "mixed":
        # the backward scatters with FP64 atomics: equal up to their rounding order
        for x, y in ((a[2], b[2]), (a[3], b[3])):
            assert float((x - y).norm() / y.norm()) <= 1e-6
    assert a[4:] == b[4:]


def test_fp32_plain_mode_and_mixed_agree(W):
    p, n, res = CASES["wave40"]
    ref = _oracle("wave40")
    from paper_2609_20964_gb300 import PREC_FP32
    rec = W(res, len(p), precision=PREC_FP32, tol_rel=1e-6, max_vcycles=60)
    sdf, _ = rec.reconstruct(_t(p), _t(n), BBOX, res)
    info = rec.info()
    err = np.abs(sdf.cpu().numpy() - ref.phi).max()
    assert err <= SDF_TOL, (err, info)
    rec.close()


def test_empty_and_degenerate_inputs(W):
    from paper_2609_20964_gb300 import STATUS_EMPTY_SURFACE, STATUS_NONFINITE_INPUT, \
        STATUS_POINT_OUTSIDE_BBOX
    rec = W(16, 100)
    empty = torch.zeros((0, 3), device="cuda", dtype=torch.float32)
    sdf, nrm = rec.reconstruct(empty, empty, BBOX, 16)
    info = rec.info()
    assert info["status"] & STATUS_EMPTY_SURFACE
    assert info["n_triangles"] == 0
    assert torch.isinf(sdf).all() and (sdf > 0).all()
    assert (nrm == 0).all()
    # a NaN point is skipped: same result as without it
    p, n = synth.sphere_cloud(80, seed=2)
    pn = np.concatenate([p, np.array([[np.nan, 0.5, 0.5]], np.float32)])
    nn = np.concatenate([n, np.array([[0, 0, 1]], np.float32)])
    a, _ = rec.reconstruct(_t(p), _t(n), BBOX, 16)
    a = a.clone()
    b, _ = rec.reconstruct(_t(pn), _t(nn), BBOX, 16)
    assert rec.info()["status"] & STATUS_NONFINITE_INPUT
    assert torch.equal(a, b)
    # a point outside the box is flagged and clamped
    po = np.concatenate([p, np.array([[1.5, 0.5, 0.5]], np.float32)])
    rec.reconstruct(_t(po), _t(nn), BBOX, 16)
    assert rec.info()["status"] & STATUS_POINT_OUTSIDE_BBOX
    rec.close()


def test_mesh_capacity_overflow_is_flagged(W):
    """More triangles than mesh_capacity: the forward flags it and stays inside
    the capped triangle, record and cube-puck buffers; the same handle then
    reconstructs a surface that fits exactly (SDF against the oracle)."""
    from paper_2609_20964_gb300 import STATUS_MESH_CAPACITY
    p, n, res = CASES["sphere24"]
    rec = W(64, len(p), mesh_capacity=4096)
    rec.reconstruct(_t(p), _t(n), BBOX, 64)
    info = rec.info()
    assert info["status"] & STATUS_MESH_CAPACITY, info
    assert info["n_triangles"] > 4096, info
    sdf, _ = rec.reconstruct(_t(p), _t(n), BBOX, res)
    info = rec.info()
    assert not info["status"] & STATUS_MESH_CAPACITY, info
    assert 0 < info["n_triangles"] <= 4096, info
    err = np.abs(sdf.cpu().numpy().astype(np.float64) - _oracle("sphere24").phi).max()
    assert err <= SDF_TOL, err
    rec.close()


def test_host_errors(W):
    from paper_2609_20964_gb300 import WgeoError
    rec = W(32, 100)
    p, n = synth.sphere_cloud(100, seed=2)
    with pytest.raises(WgeoError):
        rec.reconstruct(_t(p), _t(n), BBOX, 64)              # res over the handle's bound
    with pytest.raises(WgeoError):
        rec.reconstruct(_t(p), _t(n), np.array([0, 0, 0, 1, 0, 1], np.float32), 16)   # flat box
    with pytest.raises(WgeoError):
        rec.query(_t(synth.uniform_queries(10, 1)))          # no forward yet
    rec.close()


def test_sh_generator_and_adjoint(W):
    from paper_2609_20964_gb300 import sh_surface, sh_surface_backward
    dirs, th0, _ = synth.sh_fixed_dirs_cloud(5000)
    P, N = sh_surface(_t(th0.astype(np.float32)), _t(dirs.astype(np.float32)))
    rp, rn, _ = synth.sh_surface(th0, dirs.astype(np.float32).astype(np.float64))
    assert np.abs(P.cpu().numpy() - rp).max() < 2e-6
    assert _angle_deg(N.cpu().numpy(), rn).max() < 0.01
    rng = np.random.default_rng(0)
    dpp = rng.standard_normal((5000, 3)).astype(np.float32)
    dnn = rng.standard_normal((5000, 3)).astype(np.float32)
    rec = W(16, 10)
    d = sh_surface_backward(rec, _t(th0.astype(np.float32)), _t(dirs.astype(np.float32)), _t(dpp), _t(dnn))
    want = synth.sh_surface_vjp(th0, dirs.astype(np.float32).astype(np.float64), dpp, dnn)
    rel = np.linalg.norm(d.cpu().numpy() - want) / np.linalg.norm(want)
    assert rel < 1e-4, rel
    rec.close()


@pytest.mark.slow
def test_full_size_shbody256_sampled(W):
    # the benchmark workload (200k-point SH body, 256^3, 1M queries) in the
    # benchmark's launch configuration: bins bit-exact for all points, phi and
    # normals on sampled nodes, phi at sampled queries, against the oracle
    p, n, _ = synth.sh_body_cloud(200_000, lmax=8)
    res = 256
    rec = W(res, len(p))
    sdf, nrm = rec.reconstruct(_t(p), _t(n), BBOX, res)
    q = synth.uniform_queries(1_000_000, seed=2001)
    sq, _ = rec.query(_t(q), with_normals=False)
    info = rec.info()
    assert info["status"] == 0, info
    bins = rec.bins().cpu().numpy()
    ref = OP.forward_to_mesh(p, n, BBOX, res)
    assert np.array_equal(bins, ref.bins.astype(np.int32))
    rng = np.random.default_rng(17)
    lin = rng.choice(res ** 3, 1500, replace=False)
    ophi, _, _ = OP.sdf_at(ref, lin)
    phi = sdf.cpu().numpy().reshape(-1)
    assert np.abs(phi[lin] - ophi).max() <= SDF_TOL
    # normals on 300 sampled nodes (oracle stencil on its own exact phi)
    lin2 = lin[:300]
    on, omag = OP.normals_at(ref, lin2)
    g = nrm.cpu().numpy().reshape(3, -1)[:, lin2].T
    ok = omag >= 0.9
    assert _angle_deg(g[ok], on[ok]).max() <= ANGLE_TOL_DEG
    # queries: trilinear phi at 200 sampled queries from the oracle's phi at their corners
    from oracle import iso as OI
    qi = rng.choice(len(q), 200, replace=False)
    corners, w, _ = OI.trilinear(q[qi].astype(np.float64), ref.lo, ref.h, res)
    cl = ((corners[..., 2] * res + corners[..., 1]) * res + corners[..., 0]).reshape(-1)
    uq, inv = np.unique(cl, return_inverse=True)
    ph_u, _, _ = OP.sdf_at(ref, uq)
    oq = np.sum(w * ph_u[inv].reshape(-1, 8), axis=1)
    assert np.abs(sq.cpu().numpy()[qi] - oq).max() <= SDF_TOL
    rec.close()


@pytest.mark.slow
def test_full_size_shbody256_backward_sampled(W):
    # the benchmark body at 256^3 in the benchmark's launch configuration:
    # d_points, d_normals and d_q for phi seeds at 2,000 uniform queries (no
    # masking), element by element against the oracle's adjoint, whose exact
    # distance is evaluated only at the queries' corner nodes
    p, n, _ = synth.sh_body_cloud(200_000, lmax=8)
    res = 256
    q = synth.uniform_queries(2000, seed=2101)
    g = np.random.default_rng(78).standard_normal(len(q)).astype(np.float32)
    rec = W(res, len(p))
    rec.reconstruct(_t(p), _t(n), BBOX, res)
    Q = _t(q)
    dp, dn, dq = rec.backward(q=Q, d_sdf_q=_t(g), want_dq=True)
    assert rec.info()["status"] == 0
    ref = OP.forward_to_mesh(p, n, BBOX, res)
    OP.fill_nodes(ref, OP.query_corner_nodes(q, res, ref.lo, ref.h), max(1, min(16, os.cpu_count() or 1)))
    odp, odn, odq = OP.backward(ref, q=q, d_sdf_q=g.astype(np.float64))
    for got, want, nm in ((dp, odp, "d_points"), (dn, odn, "d_normals"), (dq, odq, "d_q")):
        _check_grad(got, want, nm)
    rec.close()


@pytest.mark.slow
def test_sphere64_sampled_against_analytic_and_oracle(W):
    # the 4,096-point sphere at 64^3: every node against |x - c| - r (bounds of
    # the discretisation), sampled nodes against the oracle's exact phi
    p, n = synth.sphere_cloud()
    res = 64
    rec = W(res, len(p))
    sdf, nrm = rec.reconstruct(_t(p), _t(n), BBOX, res)
    phi = sdf.cpu().numpy().astype(np.float64)
    h = 1.0 / res
    X = OG.node_positions(OG.grid_lo(BBOX), h, res)
    ana = np.linalg.norm(X - 0.5, axis=-1) - 0.3
    band = np.abs(ana) < 5 * h
    assert np.abs(phi - ana)[band].max() <= 0.5 * h
    ref = OP.forward_to_mesh(p, n, BBOX, res)
    lin = np.random.default_rng(3).choice(res ** 3, 3000, replace=False)
    ophi, _, _ = OP.sdf_at(ref, lin)
    assert np.abs(phi.reshape(-1)[lin] - ophi).max() <= SDF_TOL
    rec.close()


@pytest.mark.parametrize("name,res", [("shbody44", 44), ("sphere64", 64)])
def test_fp64_refinement_mode(W, name, res):
    """The native-FP64 refinement (WGEO_PREC_FP64) on a multigrid grid (44^3)
    and a spectral one (64^3): the same SDF as the float-float refinement to
    float32 rounding, within 1e-4 of the oracle, and gradient parity; a second
    call on the handle warm-starts from the float-float pair it left."""
    from paper_2609_20964_gb300 import PREC_FP64
    if name == "sphere64":
        p, n = synth.sphere_cloud(4096)
        ref = oracle.reconstruct(p, n, BBOX, res, workers=max(1, min(16, os.cpu_count() or 1)))
    else:
        p, n, _ = CASES[name]
        ref = _oracle(name)
    mixed = W(res, len(p))
    sm, _ = mixed.reconstruct(_t(p), _t(n), BBOX, res)
    sm = sm.clone()
    rec = W(res, len(p), precision=PREC_FP64, warm_start=1)
    for _ in range(2):
        s64, _ = rec.reconstruct(_t(p), _t(n), BBOX, res)
        info = rec.info()
        assert info["status"] == 0, info
        assert float((s64 - sm).abs().max()) <= 1e-6
        assert np.abs(s64.cpu().numpy().astype(np.float64) - ref.phi).max() <= SDF_TOL
    q = synth.uniform_queries(2000, seed=35)
    gs = np.random.default_rng(7).standard_normal(len(q)).astype(np.float32)
    dp, dn, _ = rec.backward(q=_t(q), d_sdf_q=_t(gs))
    odp, odn, _ = OP.backward(ref, q=q, d_sdf_q=gs.astype(np.float64))
    _check_grad(dp, odp, "d_points")
    _check_grad(dn, odn, "d_normals")
    rec.close()
    mixed.close()
