"""Serving loop on the GPU: every result is the same alone and in a mix of
concurrent requests of different sizes (bit for bit with cold solves; within
the stated tolerances when each pooled handle warm-starts from whatever it
solved last); admission respects the memory budget; an oversized request is
refused on the host; device-resident inputs produced on the caller's stream
are read after that stream's work."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _requests():
    from paper_2609_20964_gb300.serving import Request
    out = []
    rng = np.random.default_rng(3)
    for i, (res, n) in enumerate([(32, 4000), (48, 12000), (64, 20000), (32, 3000),
                                  (64, 9000), (48, 6000), (32, 15000), (64, 5000)]):
        p, nr, _ = synth.sh_body_cloud(n, lmax=6, seed=700 + i)
        q = synth.uniform_queries(5000, seed=800 + i)
        g = rng.standard_normal(len(q)).astype(np.float32) if i % 2 == 0 else None
        out.append(Request(points=p, normals=nr, res=res, queries=q, d_sdf_q=g, rid=i))
    return out


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)


def _run(reqs, budget, streams, warm_start=1):
    from paper_2609_20964_gb300.serving import Server
    srv = Server(budget, n_streams=streams, max_points=20000, warm_start=warm_start)
    futs = [srv.submit(r) for r in reqs]
    res = [f.result(timeout=120) for f in futs]
    st = srv.stats()
    srv.close()
    return res, st


def test_alone_equals_mix(lib):
    # cold solves: the forward is bit-reproducible, whatever ran before on the handle
    reqs = _requests()
    alone = []
    for r in reqs:
        out, _ = _run([r], 4 << 30, 1, warm_start=0)
        alone.append(out[0])
    mix, st = _run(reqs, 4 << 30, 4, warm_start=0)
    assert st["completed"] == len(reqs)
    for a, m in zip(alone, mix):
        assert a.rid == m.rid
        assert np.array_equal(a.sdf_q, m.sdf_q)
        if a.d_points is not None:
            rel = np.linalg.norm(a.d_points - m.d_points) / np.linalg.norm(a.d_points)
            assert rel <= 1e-6                               # FP64-atomic accumulation order only
        assert m.info["status"] == 0


def test_alone_equals_mix_with_warm_start(lib):
    # warm starts (the default): a handle's solve starts from the last body it
    # solved, so results agree to the solver's tolerance, not bit for bit
    reqs = _requests()
    alone = []
    for r in reqs:
        out, _ = _run([r], 4 << 30, 1)
        alone.append(out[0])
    mix, st = _run(reqs + reqs, 4 << 30, 4)      # every request twice: the second runs warm
    assert st["completed"] == 2 * len(reqs)
    for k, m in enumerate(mix):
        a = alone[k % len(reqs)]
        assert a.rid == m.rid and m.info["status"] == 0
        assert np.abs(a.sdf_q - m.sdf_q).max() <= 1e-4      # 1e-4 of the unit box
        if a.d_points is not None:
            for x, y in ((a.d_points, m.d_points), (a.d_normals, m.d_normals)):
                assert np.linalg.norm(x - y) <= 1e-4 * np.linalg.norm(x)
                assert np.linalg.norm(x - y, axis=1).max() <= 1e-4 * np.linalg.norm(x, axis=1).max()


def test_device_inputs_follow_the_callers_stream(lib):
    # inputs produced on the device by work enqueued on the caller's stream
    # just before submit(): the request must read them after that work
    from paper_2609_20964_gb300.serving import Request, Server
    p, n, _ = synth.sh_body_cloud(8000, seed=901)
    q = synth.uniform_queries(3000, seed=902)
    srv = Server(4 << 30, n_streams=2, max_points=20000, warm_start=0)
    want = srv.submit(Request(points=p, normals=n, res=48, queries=q, rid=0)).result(timeout=120)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        P = torch.zeros((len(p), 3), device="cuda")
        N = torch.zeros((len(n), 3), device="cuda")
        Q = torch.zeros((len(q), 3), device="cuda")
        torch.cuda._sleep(20_000_000)                 # keep the stream busy before the copies
        P.copy_(torch.from_numpy(p).cuda(non_blocking=True))
        N.copy_(torch.from_numpy(n).cuda(non_blocking=True))
        Q.copy_(torch.from_numpy(q).cuda(non_blocking=True))
        fut = srv.submit(Request(points=P, normals=N, res=48, queries=Q, want_grid=True, rid=1))
    got = fut.result(timeout=120)
    srv.close()
    assert np.array_equal(want.sdf_q, got.sdf_q)
    assert got.sdf_grid is not None and got.done_event is not None


def test_admission_under_small_budget(lib):
    from paper_2609_20964_gb300 import Reconstructor
    reqs = [r for r in _requests() if r.res == 64]
    budget = int(Reconstructor.footprint(64, 20000) * 1.5)   # room for one 64^3 workspace at a time
    out, st = _run(reqs, budget, 3)
    assert st["completed"] == len(reqs) and st["used_bytes"] <= budget
    assert all(o.info["status"] == 0 for o in out)


def test_oversized_request_refused(lib):
    from paper_2609_20964_gb300.serving import Request, Server
    srv = Server(1 << 20, n_streams=1, max_points=20000)
    p, n = synth.sphere_cloud(100)
    f = srv.submit(Request(points=p, normals=n, res=64))
    with pytest.raises(MemoryError):
        f.result(timeout=10)
    srv.close()
