"""torch.autograd wrappers of the adjoint chain (Sec. 2.5): the gradient of a
loss through sdf_query equals a direct wgeo_backward with the same seeds, and
a backward whose forward state the handle no longer holds is refused."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BBOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as g
    g.build()
    from paper_2609_20964_gb300 import Reconstructor
    torch.cuda.set_device(0)
    return Reconstructor


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_autograd_equals_direct_backward(W):
    from paper_2609_20964_gb300.autograd import sdf_query
    p, n, _ = synth.sh_body_cloud(5000, seed=41)
    q = synth.uniform_queries(2000, seed=42)
    w = np.random.default_rng(43).standard_normal(len(q)).astype(np.float32)
    rec = W(40, len(p))
    P = _t(p).requires_grad_(True)
    N = _t(n).requires_grad_(True)
    Q = _t(q).requires_grad_(True)
    phi, _ = sdf_query(P, N, Q, rec, BBOX, 40)
    (phi * _t(w)).sum().backward()
    rec2 = W(40, len(p))
    rec2.reconstruct(_t(p), _t(n), BBOX, 40, with_sdf=False, with_normals=False)
    dp, dn, dq = rec2.backward(q=_t(q), d_sdf_q=_t(w), want_dq=True)
    torch.cuda.synchronize()
    for a, b in ((P.grad, dp), (N.grad, dn), (Q.grad, dq)):
        assert float((a - b).norm() / b.norm()) <= 1e-6      # FP64-atomic accumulation order only
    rec.close()
    rec2.close()


def test_backward_after_another_forward_is_refused(W):
    from paper_2609_20964_gb300 import StaleForwardError
    from paper_2609_20964_gb300.autograd import sdf_grid, sdf_query
    p, n = synth.sphere_cloud(3000, seed=44)
    p2, n2 = synth.sphere_cloud(3000, seed=45, radius=0.25)
    q = _t(synth.uniform_queries(500, seed=46))
    rec = W(32, 3000)
    P = _t(p).requires_grad_(True)
    phi, _ = sdf_query(P, _t(n), q, rec, BBOX, 32)
    sdf_query(_t(p2), _t(n2), q, rec, BBOX, 32)        # a second forward on the same handle
    with pytest.raises(StaleForwardError):
        phi.sum().backward()
    # the grid form too
    P.grad = None
    g, _ = sdf_grid(P, _t(n), rec, BBOX, 32)
    rec.reconstruct(_t(p2), _t(n2), BBOX, 32)
    with pytest.raises(StaleForwardError):
        g.sum().backward()
    # a backward right after its own forward still runs
    phi, _ = sdf_query(P, _t(n), q, rec, BBOX, 32)
    phi.sum().backward()
    assert torch.isfinite(P.grad).all()
    rec.close()
