"""Pins for the oracle's adjoint chain (Sec. 2.5, Eqs. 35-39): central finite
differences of the FP64 forward with the central cells frozen (the
piecewise-smooth branch that the adjoint differentiates), plus invariants."""
import numpy as np
import pytest

import synth
from oracle import pipeline as PL


@pytest.fixture(scope="module")
def small_case():
    res = 16
    p, n = synth.sphere_cloud(300, seed=5)
    p = p.astype(np.float64)
    n = n.astype(np.float64)
    bbox = np.array([0, 0, 0, 1, 1, 1], np.float32)
    rng = np.random.default_rng(1)
    q = rng.random((200, 3))
    w = dict(g=rng.standard_normal((res, res, res)), gn=rng.standard_normal((3, res, res, res)),
             q=rng.standard_normal(200), qn=rng.standard_normal((200, 3)))
    rec = PL.reconstruct(p, n, bbox, res)
    return res, p, n, bbox, q, w, rec


def _loss(res, bbox, pp, nn, qq, w, bins):
    r = PL.reconstruct(pp, nn, bbox, res, frozen_bins=bins)
    sq, nq = PL.query(r, qq)
    return (np.sum(w["g"] * r.phi) + np.sum(w["gn"] * r.nrm) + np.sum(w["q"] * sq)
            + np.sum(w["qn"] * nq))


def test_full_chain_matches_central_fd(small_case):
    res, p, n, bbox, q, w, rec = small_case
    dp, dn, dq = PL.backward(rec, w["g"], w["gn"], q, w["q"], w["qn"])
    eps = 1e-6
    for i, ax in [(3, 0), (17, 2), (100, 1), (250, 0)]:
        for name, arr, g in (("x", p, dp), ("n", n, dn)):
            a1 = arr.copy()
            a2 = arr.copy()
            a1[i, ax] += eps
            a2[i, ax] -= eps
            if name == "x":
                f1 = _loss(res, bbox, a1, n, q, w, rec.bins)
                f2 = _loss(res, bbox, a2, n, q, w, rec.bins)
            else:
                f1 = _loss(res, bbox, p, a1, q, w, rec.bins)
                f2 = _loss(res, bbox, p, a2, q, w, rec.bins)
            fd = (f1 - f2) / (2 * eps)
            assert fd == pytest.approx(g[i, ax], rel=1e-6, abs=1e-6 * np.abs(g).max())
    for i, ax in [(5, 0), (50, 1), (150, 2)]:
        q1 = q.copy()
        q2 = q.copy()
        q1[i, ax] += eps
        q2[i, ax] -= eps
        fd = (_loss(res, bbox, p, n, q1, w, rec.bins) - _loss(res, bbox, p, n, q2, w, rec.bins)) / (2 * eps)
        assert fd == pytest.approx(dq[i, ax], rel=1e-6, abs=1e-6 * np.abs(dq).max())


def test_adjoint_parts_invariants(small_case):
    res, p, n, bbox, q, w, rec = small_case
    _, _, _, parts = PL.backward(rec, w["g"], None, None, None, None, return_parts=True)
    # the loss only sees chi through (chi - c) / (chi2 - chi1) and c: a uniform
    # shift of chi changes nothing, so dL/dchi sums to zero
    assert abs(parts["dchi"].sum()) < 1e-10 * np.abs(parts["dchi"]).sum()
    # lambda solves the adjoint system L lambda = dchi (Eq. 38) with zero mean
    from oracle import poisson as P
    lam = parts["lam"]
    assert np.abs(P.laplacian(lam) - parts["dchi"]).max() < 1e-9 * np.abs(parts["dchi"]).max()
    assert abs(lam.mean()) < 1e-12


def test_backward_linear_in_seeds(small_case):
    res, p, n, bbox, q, w, rec = small_case
    a = PL.backward(rec, w["g"], None)
    b = PL.backward(rec, None, w["gn"])
    ab = PL.backward(rec, w["g"], w["gn"])
    assert np.allclose(ab[0], a[0] + b[0], rtol=1e-10, atol=1e-12)
    assert np.allclose(ab[1], a[1] + b[1], rtol=1e-10, atol=1e-12)


def test_exact_query_seeds_match_central_fd(small_case):
    # the adjoint of the exact off-grid distance (Eq. 33 at arbitrary q):
    # central differences of sum g phi_exact(q) through the whole forward
    from oracle import query_exact as QE
    res, p, n, bbox, q, w, rec = small_case
    rng = np.random.default_rng(9)
    qe = rng.uniform(0.15, 0.85, (60, 3))
    ge = rng.standard_normal(60)
    dp, dn, dq = PL.backward(rec, q_exact=qe, d_sdf_exact=ge)

    def loss(pp, nn, qq):
        r = PL.forward_to_mesh(pp, nn, bbox, res, frozen_bins=rec.bins)
        return float(np.sum(ge * QE.query_exact(qq, r.mesh["verts"])[0]))

    eps = 1e-6
    for i, ax in [(3, 0), (17, 2), (100, 1), (250, 0)]:
        for arr, g, is_p in ((p, dp, True), (n, dn, False)):
            a1, a2 = arr.copy(), arr.copy()
            a1[i, ax] += eps
            a2[i, ax] -= eps
            f1 = loss(a1, n, qe) if is_p else loss(p, a1, qe)
            f2 = loss(a2, n, qe) if is_p else loss(p, a2, qe)
            assert (f1 - f2) / (2 * eps) == pytest.approx(g[i, ax], rel=1e-5, abs=1e-6 * np.abs(g).max())
    for i, ax in [(4, 0), (20, 1), (41, 2)]:
        q1, q2 = qe.copy(), qe.copy()
        q1[i, ax] += eps
        q2[i, ax] -= eps
        fd = (loss(p, n, q1) - loss(p, n, q2)) / (2 * eps)
        assert fd == pytest.approx(dq[i, ax], rel=1e-5, abs=1e-6 * np.abs(dq).max())
