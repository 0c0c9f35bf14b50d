"""Parity orientation (Sec. 2.2) on the GPU vs the oracle, through the C ABI.

Every output is an integer decision taken in float32 on both sides, so the
bar is bit-exact: r_d, the statistics (N and N_one along both directions,
the iteration flags) and the oriented normals."""
import numpy as np
import pytest

import synth
from oracle import normals_pca as D
from oracle import orient as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)


@pytest.fixture(scope="module")
def rec():
    import __graft_entry__ as g
    g.build()
    from paper_2609_20964_gb300 import Reconstructor
    torch.cuda.set_device(0)
    r = Reconstructor(16, 200_000)
    yield r
    r.close()


def _gpu(rec, P, N, bbox=BOX, gamma=2.5, n_tol=2):
    Pt = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).cuda()
    Nt = torch.from_numpy(np.ascontiguousarray(N, dtype=np.float32)).cuda()
    out, st, rd = rec.orient_normals(Pt, Nt, bbox, gamma, n_tol, with_stats=True)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy().astype(np.int64), np.float32(rd.item())


def _random_signs(N, seed):
    s = np.random.default_rng(seed).choice([-1, 1], len(N)).astype(np.float32)
    return (N * s[:, None]).astype(np.float32)


def _same(g, o):
    gn, gs, grd = g
    on, os_, ord_ = o
    assert grd == ord_, (grd, ord_)
    bad = np.nonzero((gs != os_).any(axis=1))[0]
    assert len(bad) == 0, f"stats differ at {bad[:8]}: gpu {gs[bad[:3]].tolist()} oracle {os_[bad[:3]].tolist()}"
    assert np.array_equal(gn, on)


def test_sphere_random_signs_bit_exact(rec):
    p, n = synth.sphere_cloud(3000, seed=5)
    N = _random_signs(n, 0)
    g = _gpu(rec, p, N)
    _same(g, O.orient(p, N))
    assert (np.sum(g[0] * (p - 0.5), axis=1) > 0).all()


def test_star_body_with_oracle_pca_normals(rec):
    # the oracle's own D-PCA normals (unoriented) as input to both sides
    P, Nx, _ = synth.sh_body_cloud(12_000, seed=41, noise=0.002)
    Npca, _, cnt = D.dpca_normals(P.astype(np.float64), 0.05, 5e-5)
    Npca = Npca.astype(np.float32)
    g = _gpu(rec, P, Npca)
    _same(g, O.orient(P, Npca))
    ok = cnt >= 3
    outward = np.sum(g[0][ok] * Nx[ok], axis=1) > 0
    assert outward.mean() > 0.99


def test_thin_slab_and_hand_case(rec):
    import tests.test_oracle_orient as T
    P, Nx = T._thin_slab()
    g = _gpu(rec, P, -Nx)
    _same(g, O.orient(P, -Nx))
    faces = np.abs(Nx[:, 2]) > 0.5
    assert np.array_equal(g[0][faces], Nx[faces])
    # two planes: the hand-computed statistics of (0.5, 0.5, 0)
    grid = T._grid(9, 0.125)
    Q = np.r_[np.c_[grid, np.zeros(len(grid))], np.c_[grid, np.ones(len(grid))]]
    i = int(np.argmin(np.abs(Q - [0.5, 0.5, 0.0]).sum(1)))
    N = np.zeros_like(Q, dtype=np.float32)
    N[i] = (0, 0, 1)
    gn, gs, grd = _gpu(rec, Q, N, bbox=np.array([0, 0, 0, 1, 1, 1], np.float32))
    assert grd == np.float32(0.15625)
    assert gs[i].tolist() == [1, 2, 0, 2, 9] and gn[i].tolist() == [0, 0, -1]
    assert not gs[np.arange(len(Q)) != i].any()


def test_edge_cases(rec):
    p, n = synth.sphere_cloud(800, seed=6)
    N = _random_signs(n, 1)
    N[3] = 0                                   # zero normal: left alone
    N[4] = (np.nan, 0, 0)                      # non-finite normal: left alone
    P = p.copy()
    P[5] = (np.inf, 0, 0)                      # non-finite point: not part of the cloud
    P[6] = P[7]                                # a duplicate
    N[8] *= 1e-3                               # a short normal: scaled to unit length
    want = O.orient(P, N)
    got = _gpu(rec, P, N)
    # NaN compares unequal: check that entry apart
    assert np.isnan(got[0][4, 0]) and np.isnan(want[0][4, 0])
    got[0][4] = want[0][4] = 0
    _same(got, want)
    # a box that holds part of the cloud gives the same decisions
    half = np.array([0.3, 0.3, 0.3, 0.6, 0.6, 0.6], dtype=np.float32)
    got2 = _gpu(rec, P, N, bbox=half)
    got2[0][4] = 0
    _same(got2, want)
    # fewer than two points, no points
    one = _gpu(rec, p[:1], n[:1])
    assert one[2] == 0 and not one[1].any() and np.array_equal(one[0], n[:1])
    Pt = torch.zeros((0, 3), device="cuda")
    out, st, rd = rec.orient_normals(Pt, torch.zeros((0, 3), device="cuda"), BOX, with_stats=True)
    torch.cuda.synchronize()
    assert out.shape == (0, 3) and float(rd.item()) == 0.0
    from paper_2609_20964_gb300 import WgeoError
    for kw in (dict(gamma=0.5), dict(gamma=float("inf")), dict(n_tol=-1)):
        args = dict(gamma=2.5, n_tol=2)
        args.update(kw)
        with pytest.raises(WgeoError):
            rec.orient_normals(torch.from_numpy(p).cuda(), torch.from_numpy(n).cuda(), BOX, **args)


def test_full_cloud_sampled(rec):
    # the 200,000-point star body with its analytic normals, random signs:
    # r_d over the whole cloud and the rays of sampled points against the
    # oracle; the share of outward results over all points
    P, Nx, _ = synth.sh_body_cloud()
    N = _random_signs(Nx, 2)
    gn, gs, grd = _gpu(rec, P, N)
    idx = np.random.default_rng(7).choice(len(P), 40, replace=False)
    on, os_, ord_ = O.orient(P, N, only=idx)
    assert grd == ord_
    assert np.array_equal(gs[idx], os_[idx]) and np.array_equal(gn[idx], on[idx])
    assert (np.sum(gn * Nx, axis=1) > 0).mean() > 0.999
