"""Pins for the oracle's binning, splat and divergence (Sec. 2.3, Eqs. 22-26).

Every expected value here is derived by hand from the equations, not by
re-running the oracle's formula.
"""
import numpy as np
import pytest

from oracle import divergence as D
from oracle import grid as G
from oracle import splat as SP


def test_bin_faces_and_ulps(unit_bbox):
    res = 64                        # h = 1/64 exactly
    h = G.grid_spacing(unit_bbox, res)
    assert h == 1.0 / 64
    xs, want = [], []
    for k in (1, 17, 40, 63):
        f = np.float32(k / 64.0)
        xs += [f, np.nextafter(f, np.float32(0)), np.nextafter(f, np.float32(2))]
        want += [k, k - 1, k]
    pts = np.array([[x, 0.5, 0.25] for x in xs], dtype=np.float32)
    b, finite, status = G.bin_points(pts, unit_bbox, res)
    assert finite.all() and status == 0
    assert b[:, 0].tolist() == want
    assert (b[:, 1] == 32).all() and (b[:, 2] == 16).all()


def test_bin_clamp_outside_and_nonfinite(unit_bbox):
    pts = np.array([[1.0, 0.5, 0.5], [-0.01, 0.5, 0.5], [0.5, np.nan, 0.5], [0.2, 0.2, 0.2]],
                   dtype=np.float32)
    b, finite, status = G.bin_points(pts, unit_bbox, 8)
    assert b[0, 0] == 7 and b[1, 0] == 0       # x = hi is inside the closed box, clamped to the last cell
    assert finite.tolist() == [True, True, False, True]
    assert status & G.STATUS_POINT_OUTSIDE_BBOX
    assert status & G.STATUS_NONFINITE_INPUT
    assert b[3].tolist() == [1, 1, 1]


def test_noncubic_box_spacing():
    bbox = np.array([0, 0, 0, 2, 1, 0.5], dtype=np.float32)
    assert G.grid_spacing(bbox, 16) == 2.0 / 16


def _one_point_alpha(x, res=8):
    bbox = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
    lo = G.grid_lo(bbox)
    h = G.grid_spacing(bbox, res)
    b, _, _ = G.bin_points(np.array([x], dtype=np.float32), bbox, res)
    cells, alpha, _, inside = SP.splat_weights(np.array([x], dtype=np.float64), b, lo, h, res)
    return cells[0], alpha[0], inside[0], b[0]


def test_splat_worked_example_cell_centre():
    # point at the centre of cell (3,4,2) of an 8^3 grid: unnormalised weights
    # 1/2 (centre), 1/16 (face), 1/32 (edge), 1/64 (corner), total 11/8
    res = 8
    x = [(3 + 0.5) / res, (4 + 0.5) / res, (2 + 0.5) / res]
    cells, alpha, inside, b = _one_point_alpha(x, res)
    assert b.tolist() == [3, 4, 2]
    want = {0: 4 / 11, 1: 1 / 22, 2: 1 / 44, 3: 1 / 88}
    for o in range(27):
        k = int(np.sum(np.abs(cells[o] - b)))
        assert alpha[o] == pytest.approx(want[k], rel=1e-14)
    assert alpha.sum() == pytest.approx(1.0, rel=1e-15)


def test_splat_offcentre_hand_values():
    # x = centre - h/4 along x: delta=(-1,0,0): |dx| = 3h/4 -> (1/2)(1-3/8) = 5/16,
    # transverse factors 1/2 -> 5/64; delta=(+1,0,0): |dx| = 5h/4 -> (1/2)(1-5/8) = 3/16 -> 3/64
    res = 8
    h = 1.0 / res
    x = [(3 + 0.5) * h - 0.25 * h, (4 + 0.5) * h, (2 + 0.5) * h]
    cells, alpha, inside, b = _one_point_alpha(x, res)
    bbox = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
    _, a, _ = SP.raw_weights(np.array([x]), b[None, :], G.grid_lo(bbox), h)
    idx_m = [o for o in range(27) if (cells[o] - b).tolist() == [-1, 0, 0]][0]
    idx_p = [o for o in range(27) if (cells[o] - b).tolist() == [1, 0, 0]][0]
    assert a[0, idx_m] == pytest.approx(5 / 64, rel=1e-12)
    assert a[0, idx_p] == pytest.approx(3 / 64, rel=1e-12)
    assert a[0, SP.CENTRE_INDEX] == 0.5


def test_splat_boundary_renormalises_in_grid():
    # point at the centre of corner cell (0,0,0): only the 8 in-grid cells
    # (centre 32/64, 3 faces 4/64, 3 edges 2/64, 1 corner 1/64) -> total 51/64
    res = 8
    x = [0.5 / res] * 3
    cells, alpha, inside, b = _one_point_alpha(x, res)
    assert inside.sum() == 8
    assert alpha[SP.CENTRE_INDEX] == pytest.approx(0.5 / (51 / 64), rel=1e-14)
    assert alpha[~inside].sum() == 0
    assert alpha.sum() == pytest.approx(1.0, rel=1e-15)


def test_splat_conservation(unit_bbox):
    rng = np.random.default_rng(3)
    res = 12
    p = rng.random((500, 3)).astype(np.float32)
    n = rng.standard_normal((500, 3)).astype(np.float32)
    b, fin, _ = G.bin_points(p, unit_bbox, res)
    V = SP.splat(p, n, b, fin, G.grid_lo(unit_bbox), G.grid_spacing(unit_bbox, res), res)
    assert np.allclose(V.reshape(-1, 3).sum(0), n.astype(np.float64).sum(0), rtol=0, atol=1e-10)


def test_divergence_closed_forms():
    n = 6
    V = np.zeros((n, n, n, 3))
    V[..., 0] = 1.0                                   # constant x-field
    b = D.divergence(V, remove_mean=False)
    assert np.allclose(b[:, :, 0], 1.0) and np.allclose(b[:, :, -1], -1.0)
    assert np.allclose(b[:, :, 1:-1], 0.0)
    V2 = np.zeros((n, n, n, 3))
    V2[..., 1] = np.arange(n)[None, :, None]          # V_y = y index
    b2 = D.divergence(V2, remove_mean=False)
    assert np.allclose(b2[:, 1:-1, :], 1.0)           # (V_{j+1} - V_{j-1}) / 2
    assert np.allclose(b2[:, 0, :], 0.5)              # face (0+1)/2 - 0
    assert np.allclose(b2[:, -1, :], -(n - 2 + n - 1) / 2.0)


def test_divergence_telescopes_and_adjoint():
    rng = np.random.default_rng(0)
    V = rng.standard_normal((7, 5, 6, 3))
    b = D.divergence(V, remove_mean=False)
    assert abs(b.sum()) < 1e-12
    u = rng.standard_normal((7, 5, 6))
    lhs = np.sum(D.divergence(V) * u)
    rhs = np.sum(V * D.divergence_adjoint(u))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_splat_adjoint_identity_and_fd(unit_bbox):
    rng = np.random.default_rng(4)
    res = 10
    lo = G.grid_lo(unit_bbox)
    h = G.grid_spacing(unit_bbox, res)
    p = rng.random((60, 3))
    n = rng.standard_normal((60, 3))
    b, fin, _ = G.bin_points(p.astype(np.float32), unit_bbox, res)
    W = rng.standard_normal((res, res, res, 3))
    dx, dn = SP.splat_adjoint(p, n, b, fin, lo, h, res, W)
    # linear in n: <S n, W> = <n, S^T W>
    assert np.sum(SP.splat(p, n, b, fin, lo, h, res) * W) == pytest.approx(np.sum(n * dn), rel=1e-12)
    eps = 1e-7
    for i, ax in [(0, 0), (7, 1), (33, 2)]:
        pp, pm = p.copy(), p.copy()
        pp[i, ax] += eps
        pm[i, ax] -= eps
        fd = (np.sum(SP.splat(pp, n, b, fin, lo, h, res) * W)
              - np.sum(SP.splat(pm, n, b, fin, lo, h, res) * W)) / (2 * eps)
        assert fd == pytest.approx(dx[i, ax], rel=1e-6, abs=1e-8)
