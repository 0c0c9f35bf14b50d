"""The differentiable shape-optimisation workload end to end (Sec. 2.5, last
paragraph; Sec. 3.3; loss reading R11), GPU against the FP64 oracle.

Workload: a degree-6 spherical-harmonic body (49 float32 coefficients) at
100,000 fixed seeded directions, 128^3 grid, loss = mean (phi(q) -
phi_target(q))^2 at 500,000 uniform queries, phi_target = the same pipeline
at seeded target coefficients.

* theta-gradient through the autograd chain (sh_points -> sdf_query ->
  loss.backward()) against the oracle's adjoint chained through the
  generator's VJP: relative 2-norm <= 1e-4 and every component within
  1e-4 of the largest;
* the same gradient against central finite differences of the FP64 oracle
  loss (step 1e-4, central cells frozen), stored by tests/golden/make_c3_fd.py:
  within 1e-2 along each stored direction;
* d_points and d_normals of the GPU backward on the oracle's own float32
  points with the oracle's seeds: every point within 1e-4 of the largest
  gradient and 1e-4 relative in the 2-norm.

No seed is masked: the medial-axis nodes, where the closest point jumps, are
decided on the refined (float-float) surface as the oracle decides them.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import shape_opt as SO

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

BBOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
RES = 128
GRAD_TOL = 1e-4
FD_TOL = 1e-2
HERE = os.path.dirname(os.path.abspath(__file__))
WORKERS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def case():
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    ci = synth.config_inputs("shopt128")
    dirs, th0, tht, q = ci["dirs"], ci["theta"], ci["theta_target"], ci["queries"]
    # the oracle: target and base losses, seeds, adjoint gradient
    pt, nt = SO.sh_cloud(tht, dirs)
    phi_t, _ = SO.phi_at_queries(pt, nt, q, BBOX, RES, WORKERS)
    p0, n0 = SO.sh_cloud(th0, dirs)
    phi0, rec0 = SO.phi_at_queries(p0, n0, q, BBOX, RES, WORKERS)
    seeds = SO.loss_seeds(phi0, phi_t)
    dth, dp, dn = SO.theta_gradient(th0, dirs, rec0, q, seeds)
    return dict(dirs=dirs, th0=th0, tht=tht, q=q, p0=p0, n0=n0, seeds=seeds, loss=SO.loss(phi0, phi_t),
                dth=dth, dp=dp, dn=dn)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_theta_gradient(c):
    from paper_2609_20964_gb300 import Reconstructor
    from paper_2609_20964_gb300.autograd import sdf_query, sh_points
    dirs = _t(c["dirs"].astype(np.float32))
    Q = _t(c["q"])
    rec_t = Reconstructor(RES, len(c["dirs"]))
    with torch.no_grad():
        pt, nt = sh_points(_t(c["tht"].astype(np.float32)), dirs, rec_t)
        phi_t, _ = sdf_query(pt, nt, Q, rec_t, BBOX, RES)
    rec = Reconstructor(RES, len(c["dirs"]))
    theta = _t(c["th0"].astype(np.float32)).requires_grad_(True)
    p, n = sh_points(theta, dirs, rec)
    phi, _ = sdf_query(p, n, Q, rec, BBOX, RES)
    loss = torch.mean((phi - phi_t) ** 2)
    loss.backward()
    torch.cuda.synchronize()
    out = theta.grad.double().cpu().numpy(), float(loss.detach())
    rec.close()
    rec_t.close()
    return out


def test_theta_gradient_matches_oracle_adjoint_and_fd(case):
    g, loss = _gpu_theta_gradient(case)
    want = case["dth"]
    assert loss == pytest.approx(case["loss"], rel=1e-3)
    rel = np.linalg.norm(g - want) / np.linalg.norm(want)
    assert rel <= GRAD_TOL, f"dtheta relative error {rel:.3e}"
    assert np.abs(g - want).max() <= GRAD_TOL * np.abs(want).max()
    with open(os.path.join(HERE, "golden", "c3_theta_fd.json")) as f:
        fd = json.load(f)
    for name, v, d in zip(fd["names"], fd["directions"], fd["fd"]):
        got = float(g @ np.asarray(v))
        assert abs(got - d) <= FD_TOL * abs(d), f"{name}: adjoint {got:.6e} vs FD {d:.6e}"


def test_point_gradients_elementwise(case):
    from paper_2609_20964_gb300 import Reconstructor
    rec = Reconstructor(RES, len(case["p0"]))
    rec.reconstruct(_t(case["p0"]), _t(case["n0"]), BBOX, RES, with_sdf=False, with_normals=False)
    Q = _t(case["q"])
    dp, dn, _ = rec.backward(q=Q, d_sdf_q=_t(case["seeds"].astype(np.float32)))
    torch.cuda.synchronize()
    assert rec.info()["status"] == 0
    for got, want, nm in ((dp, case["dp"], "d_points"), (dn, case["dn"], "d_normals")):
        got = got.double().cpu().numpy()
        rel = np.linalg.norm(got - want) / np.linalg.norm(want)
        per_point = np.linalg.norm(got - want, axis=1).max() / np.linalg.norm(want, axis=1).max()
        assert rel <= GRAD_TOL, f"{nm}: relative 2-norm error {rel:.3e}"
        assert per_point <= GRAD_TOL, f"{nm}: largest per-point error {per_point:.3e} of the largest gradient"
    rec.close()
