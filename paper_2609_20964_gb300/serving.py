"""Request loop with continuous batching of reconstructions of differing grid
sizes and point counts.

* A request carries a point cloud (host or device) with normals, a box, a grid
  size, optional query points and an optional adjoint seed at the queries
  (then the point/normal gradients are returned too).
* Admission: a request runs when a stream slot is free and its handle fits
  the device-memory budget.  Handles (library workspaces, sized by
  ``wgeo_footprint_bytes``) are pooled per (grid size, point-count bucket):
  a request takes a handle of the smallest bucket that holds its cloud, so
  small clouds do not reserve the workspace of the largest.  Handles are
  reused, so grids and (with ``warm_start``, on by default) the previous
  indicator stay resident and seed the next solve of that handle; idle
  handles are evicted when a new size needs room.
* Inputs may live on the host or the device.  Device inputs are read on the
  request's stream after an event recorded on the caller's current stream at
  submit(), so work the caller enqueued to produce them comes first; a
  returned SDF grid is marked as used on the caller's stream, so freeing it
  there cannot hand its memory to the request stream early.
* Requests that arrive while others are on the GPU are admitted as soon as a
  slot and memory free up; each runs on its own CUDA stream, so the kernels of
  different requests overlap on the device.
* Order: when a slot frees, the pending request with the fewest grid cells
  goes first (ties by arrival), unless the oldest has waited more than
  ``max_wait_s``; then the oldest goes.  Small grids then do not queue behind
  large ones, and no request waits without bound.
* Completion is detected with CUDA events (host polling, no device spin);
  latency = completion - arrival, reported as p50 / p99.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np
import torch

from .api import Reconstructor


@dataclass(eq=False)
class Request:
    points: object                 # [n,3] float32 (numpy or torch)
    normals: object
    res: int
    bbox: tuple = (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)
    queries: object = None         # [m,3] float32 or None
    d_sdf_q: object = None         # [m] adjoint seed at the queries (gradients requested)
    want_grid: bool = False        # return the SDF grid (device tensor)
    arrival: float = field(default_factory=time.perf_counter)
    rid: int = 0
    ready: object = None           # set by submit(): event on the caller's stream (device inputs)
    caller_stream: object = None   # set by submit(): the caller's current stream


@dataclass
class Result:
    rid: int
    sdf_q: np.ndarray | None
    d_points: np.ndarray | None
    d_normals: np.ndarray | None
    sdf_grid: torch.Tensor | None
    info: dict
    latency_s: float
    res: int = 0
    done_event: object = None      # CUDA event after the request's last kernel


class _Slot:
    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.busy = False


def _buckets(max_points: int):
    """Point-count buckets: powers of four from 16,384 up to max_points."""
    out, b = [], 16_384
    while b < max_points:
        out.append(b)
        b *= 4
    out.append(int(max_points))
    return tuple(out)


class Server:
    def __init__(self, budget_bytes: int, n_streams: int = 4, max_points: int = 500_000,
                 device=None, point_buckets=None, warm_start: int = 1, max_wait_s: float = 0.05,
                 **options):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.budget = int(budget_bytes)
        self.max_points = max_points
        self.buckets = tuple(sorted(point_buckets)) if point_buckets else _buckets(max_points)
        if self.buckets[-1] < max_points:
            raise ValueError("the largest point bucket must hold max_points")
        self.options = dict(options, warm_start=warm_start)
        self.max_wait_s = float(max_wait_s)
        self.slots = [_Slot(self.device) for _ in range(n_streams)]
        self.free_handles = collections.defaultdict(list)   # (res, bucket) -> [Reconstructor]
        self.used_bytes = 0
        self.pending = collections.deque()
        self.inflight = []
        self.latencies = []
        self.latencies_by_res = collections.defaultdict(list)
        self.completed = 0
        self.lock = threading.Condition()
        self.stop_flag = False
        self.worker = threading.Thread(target=self._run, daemon=True)
        self.worker.start()

    # ---------------------------------------------------------------- public
    def submit(self, req: Request) -> Future:
        fut = Future()
        n = int(req.points.shape[0])
        if n > self.buckets[-1]:
            fut.set_exception(ValueError(f"{n} points exceed the server's max_points {self.buckets[-1]}"))
            return fut
        need = self.footprint(req.res, self.bucket_of(n))
        if need > self.budget:
            fut.set_exception(MemoryError(
                f"a {req.res}^3 workspace for {n} points needs {need} bytes, budget is {self.budget}"))
            return fut
        req.caller_stream = torch.cuda.current_stream(self.device)
        if any(isinstance(a, torch.Tensor) and a.is_cuda
               for a in (req.points, req.normals, req.queries, req.d_sdf_q)):
            req.ready = torch.cuda.Event()
            req.ready.record(req.caller_stream)
        with self.lock:
            self.pending.append((req, fut))
            self.lock.notify()
        return fut

    def close(self):
        with self.lock:
            self.stop_flag = True
            self.lock.notify()
        self.worker.join()
        for hs in self.free_handles.values():
            for h in hs:
                h.close()
        self.free_handles.clear()

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        per = {r: {"count": len(v), "p50_ms": 1e3 * float(np.percentile(v, 50)),
                   "p99_ms": 1e3 * float(np.percentile(v, 99))}
               for r, v in sorted(self.latencies_by_res.items())}
        return {"completed": self.completed, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "used_bytes": self.used_bytes,
                "by_res": per}

    # ---------------------------------------------------------------- internals
    def bucket_of(self, n: int) -> int:
        return next(b for b in self.buckets if b >= n)

    def footprint(self, res: int, bucket: int | None = None) -> int:
        return Reconstructor.footprint(res, self.max_points if bucket is None else bucket, **self.options)

    def _take_handle(self, res: int, n: int):
        key = (res, self.bucket_of(n))
        if self.free_handles[key]:
            return self.free_handles[key].pop()
        need = self.footprint(*key)
        # evict idle handles of other kinds until the new one fits
        while self.used_bytes + need > self.budget:
            victim = None
            for k, hs in self.free_handles.items():
                if hs:
                    victim = (k, hs.pop())
                    break
            if victim is None:
                return None
            victim[1].close()
            self.used_bytes -= self.footprint(*victim[0])
        with torch.cuda.device(self.device):
            h = Reconstructor(res, key[1], device=self.device.index, **self.options)
        h.pool_key = key
        self.used_bytes += need
        return h

    def _next_index(self) -> int:
        """The pending request to run next: the oldest if it has waited more
        than max_wait_s, else the one with the fewest grid cells (then the
        earliest)."""
        if time.perf_counter() - self.pending[0][0].arrival > self.max_wait_s:
            return 0
        best, key = 0, None
        for i, (r, _) in enumerate(self.pending):
            k = (r.res, r.arrival)
            if key is None or k < key:
                best, key = i, k
        return best

    def _launch(self, req: Request, fut: Future, slot: _Slot, h: Reconstructor):
        dev = self.device
        if req.ready is not None:
            slot.stream.wait_event(req.ready)
        with torch.cuda.stream(slot.stream):
            def to_dev(a):
                if a is None:
                    return None
                t = torch.as_tensor(a)
                return t.to(dev, non_blocking=True).contiguous() if t.device != dev else t.contiguous()
            P = to_dev(req.points)
            N = to_dev(req.normals)
            Q = to_dev(req.queries)
            G = to_dev(req.d_sdf_q)
            sdf, _ = h.reconstruct(P, N, req.bbox, req.res, with_sdf=req.want_grid, with_normals=False,
                                   stream=slot.stream)
            out = {"sdf_grid": sdf}
            if Q is not None:
                sq, _ = h.query(Q, with_normals=False, stream=slot.stream)
                out["sdf_q"] = sq.to("cpu", non_blocking=True) if Q is not None else None
                if G is not None:
                    dp, dn, _ = h.backward(q=Q, d_sdf_q=G, stream=slot.stream)
                    out["d_points"] = dp.to("cpu", non_blocking=True)
                    out["d_normals"] = dn.to("cpu", non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
            keep = (P, N, Q, G)          # inputs stay alive until the stream has used them
        self.inflight.append((req, fut, slot, h, ev, out, keep))

    def _poll(self):
        done = []
        for item in self.inflight:
            if item[4].query():
                done.append(item)
        gone = {id(item) for item in done}
        self.inflight = [item for item in self.inflight if id(item) not in gone]
        for item in done:
            req, fut, slot, h, ev, out, _ = item
            info = h.info()
            lat = time.perf_counter() - req.arrival
            self.latencies.append(lat)
            self.latencies_by_res[req.res].append(lat)
            self.completed += 1
            grid = out["sdf_grid"]
            if grid is not None and req.caller_stream is not None:
                grid.record_stream(req.caller_stream)
            res = Result(rid=req.rid,
                         sdf_q=out["sdf_q"].numpy() if out.get("sdf_q") is not None else None,
                         d_points=out["d_points"].numpy() if "d_points" in out else None,
                         d_normals=out["d_normals"].numpy() if "d_normals" in out else None,
                         sdf_grid=grid, info=info, latency_s=lat, res=req.res, done_event=ev)
            slot.busy = False
            self.free_handles[h.pool_key].append(h)
            fut.set_result(res)
        return bool(done)

    def _run(self):
        torch.cuda.set_device(self.device)
        while True:
            with self.lock:
                if self.stop_flag and not self.pending and not self.inflight:
                    return
            progressed = self._poll()
            with self.lock:
                while self.pending:
                    slot = next((s for s in self.slots if not s.busy), None)
                    if slot is None:
                        break
                    pick = self._next_index()
                    req, fut = self.pending[pick]
                    h = self._take_handle(req.res, int(req.points.shape[0]))
                    if h is None:
                        break           # memory: wait for a running request to finish
                    del self.pending[pick]
                    slot.busy = True
                    try:
                        self._launch(req, fut, slot, h)
                    except Exception as exc:  # noqa: BLE001
                        slot.busy = False
                        self.free_handles[h.pool_key].append(h)
                        fut.set_exception(exc)
                    progressed = True
                if not progressed:
                    self.lock.wait(timeout=0.0005)
