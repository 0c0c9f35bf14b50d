"""Warm-started solves on the moving-boundary workload (Sec. 3.2: the SDF is
regenerated at every step of a moving body): the travelling-wave ellipsoid,
re-sampled each step, on a grid whose solve runs the multigrid refinement
(96^3: not a power of two).  Starting the solve from the previous step's
indicator must give the same signed distance as a cold start (within 1e-4 of
the box extent, against the oracle too) in fewer refinement steps."""
import numpy as np
import pytest

import oracle
import synth
from oracle import pipeline as OP

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BBOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
SDF_TOL = 1e-4


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_2609_20964_gb300 import Reconstructor
    torch.cuda.set_device(0)
    return Reconstructor


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_warm_start_matches_cold_in_fewer_steps(W):
    res, npts = 96, 20_000
    clouds = [synth.wave_ellipsoid_cloud(t, n=npts) for t in range(4)]
    warm = W(res, npts, warm_start=1)
    cold = W(res, npts, warm_start=0)
    steps_w, steps_c = [], []
    for t, (p, n) in enumerate(clouds):
        sw, _ = warm.reconstruct(_t(p), _t(n), BBOX, res, with_normals=False)
        sw = sw.clone()
        iw = warm.info()
        sc, _ = cold.reconstruct(_t(p), _t(n), BBOX, res, with_normals=False)
        ic = cold.info()
        assert iw["status"] == 0 and ic["status"] == 0, (iw, ic)
        assert float((sw - sc).abs().max()) <= SDF_TOL
        steps_w.append(iw["solver_steps"])
        steps_c.append(ic["solver_steps"])
    # the first warm solve has nothing to start from: it is a cold one
    assert steps_w[0] == steps_c[0]
    assert sum(steps_w[1:]) < sum(steps_c[1:]), (steps_w, steps_c)
    # the last warm-started field against the oracle on sampled nodes
    p, n = clouds[-1]
    ref = OP.forward_to_mesh(p, n, BBOX, res)
    lin = np.random.default_rng(6).choice(res ** 3, 1500, replace=False)
    ophi, _, _ = OP.sdf_at(ref, lin)
    assert np.abs(sw.cpu().numpy().reshape(-1)[lin] - ophi).max() <= SDF_TOL
    warm.close()
    cold.close()


def test_warm_start_after_a_different_grid_is_cold(W):
    # the previous indicator is used only when the grid matches
    p, n = synth.wave_ellipsoid_cloud(5, n=8000)
    rec = W(48, 8000, warm_start=1)
    rec.reconstruct(_t(p), _t(n), BBOX, 40, with_normals=False)
    s1, _ = rec.reconstruct(_t(p), _t(n), BBOX, 48, with_normals=False)
    i1 = rec.info()
    ref = oracle.reconstruct(p, n, BBOX, 48, with_normals=False)
    assert np.abs(s1.cpu().numpy().astype(np.float64) - ref.phi).max() <= SDF_TOL
    cold = W(48, 8000)
    cold.reconstruct(_t(p), _t(n), BBOX, 48, with_normals=False)
    assert cold.info()["solver_steps"] == i1["solver_steps"]
    rec.close()
    cold.close()
