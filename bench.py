"""Benchmark of the SDF + normal reconstruction path on one GB300 (or N replicas).

Workload (N = 1): the 256^3 spherical-harmonic body — 200,000 area-uniform
surface points of r(u) = 0.3 + sum_{l<=8} theta_k Y_k(u), theta ~ N(0, 0.02^2),
analytic normals, position noise N(0, 0.002^2) — with 1,000,000 uniform query
points.  One step = the whole path on that input: splat, divergence,
mixed-precision Poisson solve, iso-value, marching cubes, exact SDF, stencil
normals, query at 1M points, and the adjoint of a loss on the queried SDF
(query / distance / marching-cubes / iso-value adjoints, adjoint solve, splat
adjoint).  Metric: grid cells per second (res^3 / step time).

Arms: default = the CUDA library through its C ABI; --impl reference = the
FP64 CPU oracle on the host cores (a bounded sample of the same step).
Multi-GPU: independent replicas, one per rank, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RES = 256
NPTS = 200_000
NQ = 1_000_000
BBOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)
L2_BYTES = 129 * 2 ** 20
HANDLE_OPTS = {}          # extra handle options (profiler runs only)
METRIC = "SDF+normal cells/s at 256^3 (fwd, fwd+adjoint) vs FP32 plain; p50/p99 latency"


def workload():
    import synth
    p, n, info = synth.sh_body_cloud(NPTS, lmax=8)
    q = synth.uniform_queries(NQ, seed=2001)
    # a fixed seeded adjoint seed for the queried SDF (stands in for dL/dphi(q))
    g = np.random.default_rng(2002).standard_normal(NQ).astype(np.float32) / NQ
    return p, n, q, g


# --------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        sm = []
        mx = None
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx = float(s[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if s[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- helpers
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time_ms(local_ms: float, ws: int, device) -> float:
    """The whole job's time of a timed region: the slowest rank's (every rank
    timed the same region between barriers; at N = 1, this rank's own)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, cells_per_step: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: every rank's cells over the slowest rank's time."""
    return ws * cells_per_step * steps / (total_ms / 1e3)


# --------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__ as ge
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    ge.build()
    from paper_2609_20964_gb300 import PREC_FP32, Reconstructor

    p, n, q, g = workload()
    P = torch.from_numpy(p).cuda()
    Nn = torch.from_numpy(n).cuda()
    Q = torch.from_numpy(q).cuda()
    G = torch.from_numpy(g).cuda()
    from paper_2609_20964_gb300 import _lib as L
    lib = L.load()
    # stage_timing = 1: CUDA events around each stage on the launching stream,
    # read back after the timed region (the dominant kernel's live duration)
    rec = Reconstructor(RES, NPTS, stage_timing=1, **HANDLE_OPTS)
    stream = torch.cuda.current_stream()
    N = RES ** 3

    def step():
        rec.reconstruct(P, Nn, BBOX, RES, with_sdf=True, with_normals=True, sdf_out=sdf_buf, nrm_out=nrm_buf)
        rec.query(Q, with_normals=False)
        rec.backward(q=Q, d_sdf_q=G)

    sdf_buf = torch.empty((RES, RES, RES), device="cuda")
    nrm_buf = torch.empty((3, RES, RES, RES), device="cuda")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = rec.info()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    rec.stage_times(reset=True)
    launches0 = lib.wgeo_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_ms = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.nvtx.range_push("timed")   # the profiler's launch list covers this range
    e0.record(stream)
    ev[0].record(stream)
    for k in range(args.steps):
        step()
        ev[k + 1].record(stream)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = lib.wgeo_kernel_launches() - launches0
    clocks.stop()
    st_timed = rec.stage_times(reset=True)
    timed_stage_ms = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in st_timed.items()}
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = job_time_ms(e0.elapsed_time(e1), ws, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_rate(ws, N, args.steps, total_ms)

    # forward-only rates (mixed and plain FP32) on the same input
    def time_it(fn, k):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    fwd_ms = time_it(lambda: rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf), 5)
    rec32 = Reconstructor(RES, NPTS, precision=PREC_FP32, keep_for_backward=0, max_vcycles=60, **HANDLE_OPTS)
    fwd32_ms = time_it(lambda: rec32.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf), 5)
    info32 = rec32.info()
    sdf32 = sdf_buf.clone()
    rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf)
    torch.cuda.synchronize()
    fp32_vs_mixed = float((sdf32 - sdf_buf).abs().max().item())
    sdf_mixed = sdf_buf.clone()
    rec32.close()

    # per-stage device times (CUDA events on the library's stream), separate pass
    rec_t = Reconstructor(RES, NPTS, stage_timing=2, **HANDLE_OPTS)
    for _ in range(2):
        rec_t.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf)
        rec_t.query(Q, with_normals=False)
        rec_t.backward(q=Q, d_sdf_q=G)
    torch.cuda.synchronize()
    rec_t.stage_times(reset=True)
    for _ in range(args.stage_steps):
        rec_t.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf)
        rec_t.query(Q, with_normals=False)
        rec_t.backward(q=Q, d_sdf_q=G)
    torch.cuda.synchronize()
    st = rec_t.stage_times(reset=True)
    stages = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in st.items()}
    info_t = rec_t.info()
    rec_t.close()

    # end to end through the C ABI with host buffers (pinned), copies in the timed region
    ph = torch.from_numpy(p).pin_memory()
    nh = torch.from_numpy(n).pin_memory()
    qh = torch.from_numpy(q).pin_memory()
    gh = torch.from_numpy(g).pin_memory()
    dph = torch.empty((NPTS, 3), dtype=torch.float32).pin_memory()
    dnh = torch.empty((NPTS, 3), dtype=torch.float32).pin_memory()
    Pd = torch.empty_like(P)
    Nd = torch.empty_like(Nn)
    Qd = torch.empty_like(Q)
    Gd = torch.empty_like(G)

    def e2e_step():
        Pd.copy_(ph, non_blocking=True)
        Nd.copy_(nh, non_blocking=True)
        Qd.copy_(qh, non_blocking=True)
        Gd.copy_(gh, non_blocking=True)
        rec.reconstruct(Pd, Nd, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf)
        rec.query(Qd, with_normals=False)
        dp, dn, _ = rec.backward(q=Qd, d_sdf_q=Gd)
        dph.copy_(dp, non_blocking=True)
        dnh.copy_(dn, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    ke = max(3, args.steps // 2)
    barrier()
    a.record(stream)
    for _ in range(ke):
        e2e_step()
    b.record(stream)
    barrier()
    e2e_ms = job_time_ms(a.elapsed_time(b), ws, "cuda") / ke
    h2d = (p.nbytes + n.nbytes + q.nbytes + g.nbytes)
    d2h = 2 * NPTS * 3 * 4

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_nodes)
    # roofline of the dominant kernel, on the stage times of the timed region
    hbm, peak_kind = load_peaks()
    dom = max(timed_stage_ms, key=lambda k: timed_stage_ms[k])
    roof = roofline(dom, timed_stage_ms, info, hbm, peak_kind,
                    cpu["alg_tests_per_node"] if cpu else None)

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "cells/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "SH body (degree<=8) 200k points, 256^3 grid, 1M queries, "
                               "forward + query + adjoint", "res": RES, "points": NPTS,
                   "queries": NQ, "precision": "mixed: FP32 multigrid V-cycles inside float-float "
                                                        "defect-correction refinement",
                   "l2": "working set > 1 GB per step (fields of 67 MB) exceeds the 129 MB L2; no flush",
                   "parallelism": f"replicas x{ws}",
                   "override": (RES, NPTS, NQ) != (256, 200_000, 1_000_000) or bool(HANDLE_OPTS)},
        "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99))},
        "fwd_cells_per_s": N / (fwd_ms / 1e3),
        "fwd_ms": fwd_ms,
        "fp32_plain_fwd_cells_per_s": N / (fwd32_ms / 1e3),
        "fp32_plain": {"fwd_ms": fwd32_ms, "vcycles": info32["solver_steps"],
                       "residual_rel": info32["residual_rel"],
                       "max_abs_sdf_diff_vs_mixed": fp32_vs_mixed},
        "points_per_s": NPTS / (ms_per_step / 1e3),
        "solver": {"steps": info["solver_steps"], "residual_rel": info["residual_rel"],
                   "bwd_steps": info_t["backward_steps"], "bwd_residual_rel": info_t["backward_residual_rel"]},
        "triangles": info["n_triangles"],
        "sdf_search": {"node_visits_per_warp_launch": info_t["sdf_node_visits"],
                       "leaf_visits": info_t["sdf_leaf_visits"],
                       "tri_tests": info_t["sdf_tri_tests"],
                       "tri_tests_per_node": info_t["sdf_tri_tests"] / N,
                       "near_tie_nodes": info_t["sdf_tie_nodes"]},
        "stage_ms": stages,
        "e2e": {"value": job_rate(ws, N, 1, e2e_ms), "unit": "cells/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / args.steps,
        "timed_stage_ms": timed_stage_ms,
        "roofline": roof,
        "clocks": clocks.summary(),
    }
    if rank == 0 and ws == 1 and args.serving_requests > 0:
        out["serving"] = serving_bench(args.serving_requests, value)
    if rank == 0 and args.pca_reps > 0:
        out["galerkin_q1"] = galerkin_q1_bench(Reconstructor, P, Nn, Q, G, sdf_mixed, args.pca_reps)
        out["exact_query"] = exact_query_bench(rec, P, Nn, Q, args.pca_reps)
        out["normal_estimation"] = normal_estimation_bench(rec, P, args.pca_reps, cpu is not None)
        out["normal_orientation"] = orientation_bench(rec, P, n, args.pca_reps)
    if cpu is not None:
        # SDF error of both precisions against the oracle's exact distance on its sampled nodes
        lin, ophi = cpu.pop("_sample")
        idx = torch.from_numpy(lin.astype(np.int64)).cuda()
        extent = float(np.max(BBOX[3:] - BBOX[:3]))
        err = {}
        for nm, f in (("mixed", sdf_mixed), ("fp32_plain", sdf32)):
            got = f.reshape(-1)[idx].double().cpu().numpy()
            err[nm] = float(np.abs(got - ophi).max() / extent)
        out["sdf_err_vs_oracle"] = {"max_abs_over_extent": err, "nodes": int(len(lin)),
                                    "bound": 1e-4}
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out))
    rec.close()
    if ws > 1:
        dist.destroy_process_group()


# Algorithmic bytes per cell (minimal traffic of each stage, see the design notes)
ALG_BYTES = {
    "splat": 4.0,          # write b
    "normals": 16.0,       # read phi, write 3 normal planes
    "query": 0.0,
}

# FP32 ALU peak of one GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FLOPS_PER_TRI_TEST = 40.0      # FP32 operations of one point-triangle distance
STAGE_KERNEL = {"sdf": ("sdf_kernel", "paper_2609_20964_gb300/csrc/surface.cu")}


def source_digest(rel_paths):
    import hashlib
    h = hashlib.sha256()
    for rp in rel_paths:
        with open(os.path.join(ROOT, rp), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def kernel_traffic(kernel: str, src: str):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, or None
    when the summary is missing or the kernel's sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)[kernel]
    except (OSError, KeyError, ValueError):
        return None
    srcs = [src, "paper_2609_20964_gb300/csrc/wgeo_internal.cuh"]
    if d.get("source_digest") != source_digest(srcs):
        return None
    return float(d["dram_bytes_per_launch"])


def roofline(dom, stages, info, hbm, peak_kind, alg_tests_per_node):
    N = RES ** 3
    ms = stages[dom]
    if dom == "sdf":
        # ALU-bound search; algorithmic work = triangles whose box lower bound is
        # below the node's exact distance (measured by the oracle on sampled nodes)
        kernel, src = STAGE_KERNEL[dom]
        achieved = frac = alg = None
        if alg_tests_per_node is not None and ms > 0:
            alg = alg_tests_per_node * N * FLOPS_PER_TRI_TEST
            achieved = alg / (ms / 1e3) / 1e12
            frac = achieved / FP32_PEAK_TFLOPS
        return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": frac, "traffic": kernel_traffic(kernel, src),
                "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "alg_flops_per_launch": alg, "alg_tests_per_node": alg_tests_per_node,
                "flops_per_test": FLOPS_PER_TRI_TEST, "launch_ms": ms}
    if dom in ("solve", "bwd_solve"):
        # per refinement step: residual (read chi 8 + b 4, write r 4), correction
        # update (read e 4 + chi 8, write chi 8) and per V-cycle on the fine grid
        # 2+2 RB sweeps (read x, b + write x: 12 B each) + restriction read (8 B) +
        # prolongation (read 4 + write 4)
        steps = max(info["solver_steps"], 1)
        per_step = 16 + 20 + 2 * (4 * 12 + 8 + 8) * 8 / 7
        alg = N * per_step * steps
        return {"bound": "hbm", "kernel": f"{dom} (multigrid + refinement)",
                "achieved": alg / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": alg / (ms / 1e3) / 1e9 / hbm, "traffic": None,
                "peak_kind": peak_kind, "alg_bytes_per_launch": alg}
    alg = N * ALG_BYTES.get(dom, 4.0)
    return {"bound": "hbm", "kernel": dom, "achieved": alg / (ms / 1e3) / 1e9, "peak": hbm,
            "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / hbm, "traffic": None,
            "peak_kind": peak_kind}


# ------------------------------------------------------------ unlumped Galerkin
def galerkin_q1_bench(Reconstructor, P, Nn, Q, G, sdf_lumped, reps: int):
    """The same forward, and forward + query + adjoint, with the unlumped
    27-point Galerkin operator (option galerkin = 1), CUDA events around each
    step; the solver's steps and the largest SDF difference from the lumped
    7-point result on the same cloud."""
    import torch
    rec = Reconstructor(RES, NPTS, galerkin=1, **HANDLE_OPTS)
    sdf = torch.empty((RES, RES, RES), device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()

    def fwd():
        rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf, with_normals=False)

    def step():
        rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf, with_normals=False)
        rec.query(Q, with_normals=False)
        rec.backward(q=Q, d_sdf_q=G)

    out = {}
    for name, fn in (("fwd", fwd), ("fwd_query_adjoint", step)):
        for _ in range(3):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms"] = statistics.median(a.elapsed_time(b) for a, b in ev)
    fwd()
    info = rec.info()
    N = RES ** 3
    out.update({"fwd_cells_per_s": N / (out["fwd_ms"] / 1e3),
                "step_cells_per_s": N / (out["fwd_query_adjoint_ms"] / 1e3),
                "solver_steps": info["solver_steps"], "residual_rel": info["residual_rel"],
                "status": info["status"],
                "max_abs_sdf_diff_vs_lumped": float((sdf - sdf_lumped).abs().max())})
    rec.close()
    return out


# ---------------------------------------------------------------- exact queries
def exact_query_bench(rec, P, Nn, Q, reps: int):
    """Exact off-grid signed distance and gradient at the workload's queries
    on its reconstruction (CUDA events around each call), beside the
    interpolated query of the same points."""
    import torch
    rec.reconstruct(P, Nn, BBOX, RES, with_sdf=False, with_normals=False)
    for _ in range(3):
        rec.query_exact(Q)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        rec.query_exact(Q)
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    se, _ = rec.query_exact(Q, with_grad=False)
    si, _ = rec.query(Q, with_normals=False)
    torch.cuda.synchronize()
    m = int(Q.shape[0])
    return {"queries_per_s": m / (ms / 1e3), "ms": ms, "queries": m,
            "max_abs_exact_minus_interpolated": float((se - si).abs().max())}


# --------------------------------------------------------- normal estimation
PCA_RADIUS = 0.1               # the paper's default neighbourhood radius (unit box)
FLOPS_PER_PAIR = 33.0          # FP32 operations per (point, neighbour) pair: distance,
                               # weight, first and second weighted moments


def normal_estimation_bench(rec, P, reps: int, with_oracle: bool):
    """D-PCA normals of the workload's cloud at R = 0.1 (inputs resident, CUDA
    events around each call on the launching stream)."""
    import torch
    eps = 1e-3 * PCA_RADIUS
    nrm = torch.empty_like(P)
    nrm_cnt, cnt = rec.estimate_normals(P, BBOX, PCA_RADIUS, eps, with_counts=True)
    torch.cuda.synchronize()
    pairs = int(cnt.long().sum())
    for _ in range(3):
        rec.estimate_normals(P, BBOX, PCA_RADIUS, eps, normals_out=nrm)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    l0 = rec.lib.wgeo_kernel_launches()
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        rec.estimate_normals(P, BBOX, PCA_RADIUS, eps, normals_out=nrm)
        b.record(stream)
    torch.cuda.synchronize()
    launches = rec.lib.wgeo_kernel_launches() - l0
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    n = int(P.shape[0])
    achieved = pairs * FLOPS_PER_PAIR / (ms / 1e3) / 1e12
    out = {"points_per_s": n / (ms / 1e3), "ms": ms, "points": n, "radius": PCA_RADIUS, "eps": eps,
           "mean_neighbours": pairs / n, "reps": reps, "gpu_launches_per_call": launches / reps,
           "same_as_first_call": bool(torch.equal(nrm, nrm_cnt)),
           "roofline": {"bound": "alu", "kernel": "dpca_normal_kernel (whole call timed)",
                        "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                        "alg_flops_per_launch": pairs * FLOPS_PER_PAIR, "flops_per_pair": FLOPS_PER_PAIR,
                        "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}}
    if with_oracle:
        # the oracle on a bounded sample of points (each over the whole cloud)
        from oracle import normals_pca as D
        p64 = P.double().cpu().numpy()
        p32 = P.cpu().numpy()
        idx = np.random.default_rng(9).choice(n, 64, replace=False)
        allj = np.arange(n)
        t0 = time.perf_counter()
        for i in idx:
            nb = D.in_ball_f32(p32, i, allj, PCA_RADIUS)
            D.dpca_point(p64[i], p64[nb], eps)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": len(idx) / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
                               "sample": f"{len(idx)} points, each against the whole {n}-point cloud"}
    return out


def orientation_bench(rec, P, n_exact, reps: int):
    """Parity orientation (gamma 2.5, N_tol 2) of the workload's cloud from its
    analytic normals with seeded random signs, and of the D-PCA normals
    (R = 0.1); CUDA events around each call; the share of results that point
    the analytic way."""
    import torch
    Nx = torch.from_numpy(n_exact).cuda()
    sgn = torch.from_numpy(np.random.default_rng(11).choice([-1.0, 1.0], len(n_exact)).astype(np.float32)).cuda()
    N0 = Nx * sgn[:, None]
    N = N0.clone()
    for _ in range(3):
        N.copy_(N0)
        rec.orient_normals(P, N, BBOX)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        N.copy_(N0)
        a.record(stream)
        rec.orient_normals(P, N, BBOX)
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    _, st, rd = rec.orient_normals(P, N0.clone(), BBOX, with_stats=True)
    N.copy_(N0)
    rec.orient_normals(P, N, BBOX)
    outward = float(((N * Nx).sum(1) > 0).float().mean())
    # the paper's preprocessing from raw points: D-PCA, then orientation
    Npca, _ = rec.estimate_normals(P, BBOX, PCA_RADIUS)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    rec.estimate_normals(P, BBOX, PCA_RADIUS, normals_out=Npca)
    rec.orient_normals(P, Npca, BBOX)
    t1.record(stream)
    torch.cuda.synchronize()
    ok = Npca.abs().sum(1) > 0
    pca_out = float(((Npca * Nx).sum(1)[ok] > 0).float().mean())
    st = st.cpu().numpy()
    return {"points_per_s": len(n_exact) / (ms / 1e3), "ms": ms, "gamma": 2.5, "n_tol": 2,
            "r_d": float(rd.item()), "outward_share_from_random_signs": outward,
            "mean_crossings": {"plus": float(st[:, 0].mean()), "minus": float(st[:, 2].mean())},
            "raw_points_to_oriented_normals_ms": t0.elapsed_time(t1),
            "outward_share_from_dpca": pca_out}


# --------------------------------------------------------------------- serving
def _rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def serving_bench(n_req: int, step_cells_per_s: float, load: float = 0.7):
    """The serving request mix through the request loop: grid sizes {64, 128,
    256} w.p. {0.5, 0.35, 0.15}, point counts log-uniform in [1e4, 5e5], half
    of the requests with gradients, exponential inter-arrival gaps at `load`
    times the capacity estimated from the benchmark step.  Point clouds: one
    seeded degree-8 SH body of 5e5 points; request i takes its first n_i points
    rotated about the body centre by a rotation seeded with its id.  Latency =
    completion - scheduled arrival (queueing included)."""
    import torch
    import synth
    from paper_2609_20964_gb300.serving import Request, Server
    mix = synth.serving_requests(n_req)
    bp, bn, _ = synth.sh_body_cloud(500_000, lmax=8, seed=50_000)
    c = np.array([0.5, 0.5, 0.5])
    nq = 50_000
    reqs = []
    for r in mix:
        rng = np.random.default_rng(r["seed"])
        R = _rotation(rng)
        n = min(r["n"], len(bp))
        pts = ((bp[:n].astype(np.float64) - c) @ R.T + c).astype(np.float32)
        nrm = (bn[:n].astype(np.float64) @ R.T).astype(np.float32)
        q = rng.random((nq, 3)).astype(np.float32)
        g = (rng.standard_normal(nq) / nq).astype(np.float32) if r["grad"] else None
        reqs.append((r, torch.from_numpy(pts).pin_memory(), torch.from_numpy(nrm).pin_memory(),
                     torch.from_numpy(q).pin_memory(), None if g is None else torch.from_numpy(g).pin_memory()))
    mean_cells = float(np.mean([r["res"] ** 3 for r in mix]))
    rate = load * step_cells_per_s / mean_cells          # requests per second
    srv = Server(budget_bytes=32 << 30, n_streams=4, max_points=500_000)
    # warm-up: one request per grid size (workspaces allocated, solver graphs recorded)
    warm = []
    for res in (64, 128, 256):
        r, P, N, Q, G = next(x for x in reqs if x[0]["res"] == res)
        warm.append(srv.submit(Request(points=P, normals=N, res=res, queries=Q, d_sdf_q=G)))
    for f in warm:
        f.result()
    srv.latencies.clear()
    depth = []
    futs = []
    t0 = time.perf_counter()
    t_arr = t0
    for r, P, N, Q, G in reqs:
        t_arr += r["gap"] / rate
        while time.perf_counter() < t_arr:
            time.sleep(0.0002)
        depth.append(len(srv.pending) + len(srv.inflight))
        futs.append(srv.submit(Request(points=P, normals=N, res=r["res"], queries=Q, d_sdf_q=G,
                                       arrival=t_arr, rid=r["id"])))
    results = [f.result() for f in futs]
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([x.latency_s for x in results]) * 1e3
    cells = sum(r["res"] ** 3 for r in mix)
    points = sum(min(r["n"], len(bp)) for r in mix)
    return {"requests": n_req, "offered_rate_per_s": rate, "offered_load": load,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "cells_per_s": cells / wall, "points_per_s": points / wall,
            "wall_s": wall, "queue_depth_max": int(max(depth)), "queue_depth_mean": float(np.mean(depth)),
            "streams": 4, "with_gradients": int(sum(r["grad"] for r in mix)),
            "clouds": "one seeded degree-8 SH body of 5e5 points, per-request subset and seeded rotation",
            "queries_per_request": nq}


# --------------------------------------------------------------------- oracle
def box_candidates(nodes, verts, d):
    """Per node, the triangles whose bounding-box lower bound is below the node's
    exact distance d: the work any exact box-pruned search must do."""
    lo = verts.min(axis=1)
    hi = verts.max(axis=1)
    out = np.empty(len(nodes), dtype=np.int64)
    for i, x in enumerate(nodes):
        gap = np.maximum(np.maximum(lo - x, x - hi), 0.0)
        out[i] = int(np.count_nonzero(np.einsum("ij,ij->i", gap, gap) < d[i] * d[i]))
    return out


def oracle_step(p, n, q, g, node_sample: int, rng, point_frac: float = 1.0, count_nodes: int = 0):
    """One step of the oracle on the bench workload, with the per-node distance
    search and the query stages on a random sample (and, if point_frac < 1, the
    per-point splat and splat adjoint on that fraction of the points, scaled);
    returns (estimated seconds for the full step, detail dict)."""
    from oracle import divergence as D
    from oracle import grid as OG
    from oracle import iso as OI
    from oracle import mc as OM
    from oracle import pipeline as OP
    from oracle import poisson as OPo
    from oracle import splat as OS
    N = RES ** 3
    t = {}
    lo = OG.grid_lo(BBOX)
    h = OG.grid_spacing(BBOX, RES)
    pp = p.astype(np.float64)
    nn = n.astype(np.float64)
    bins, fin, _ = OG.bin_points(pp, BBOX, RES)
    m = len(pp) if point_frac >= 1.0 else max(1, int(len(pp) * point_frac))
    t0 = time.perf_counter()
    Vs = OS.splat(pp[:m], nn[:m], bins[:m], fin[:m], lo, h, RES)
    t["splat_est"] = (time.perf_counter() - t0) * len(pp) / m
    # the global stages' cost does not depend on the values of V; with a point
    # sample, the sample's splat (the same body, fewer points) stands in for it
    V = Vs
    t0 = time.perf_counter()
    b = D.divergence(V)
    t["div"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    chi = OPo.solve(b)
    t["solve"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    c = OI.isovalue(chi, pp, fin, lo, h, RES)
    mesh = OM.marching_cubes(chi, c, lo, h)
    t["iso_mc"] = time.perf_counter() - t0
    rec = OP.Reconstruction(res=RES, h=h, lo=lo, points=pp, normals_in=nn, bins=bins, finite=fin,
                            status=0, V=V, b=b, chi=chi, c=c, mesh=mesh)
    # distance + sign on sampled nodes, extrapolated to all N nodes
    lin = rng.choice(N, node_sample, replace=False)
    t0 = time.perf_counter()
    phi_s, dist, _ = OP.sdf_at(rec, lin)
    t["sdf_sample"] = time.perf_counter() - t0
    t["sdf_est"] = t["sdf_sample"] * N / node_sample
    # stencil normals cost ~ one more distance per node in the oracle's own form: counted as 0
    # query + adjoints: adjoint solve (full), splat adjoint, iso adjoint
    t0 = time.perf_counter()
    lam = OPo.solve(chi)          # same operator and cost as the adjoint solve of dL/dchi
    t["adj_solve"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    dV = D.divergence_adjoint(lam)
    OS.splat_adjoint(pp[:m], nn[:m], bins[:m], fin[:m], lo, h, RES, dV)
    t["splat_adjoint_est"] = (time.perf_counter() - t0) * len(pp) / m
    # trilinear query at the 1M points (vectorised, measured on a tenth, scaled)
    qs = q[: len(q) // 10].astype(np.float64)
    t0 = time.perf_counter()
    OI.trilinear(qs, lo, h, RES)
    t["query_est"] = (time.perf_counter() - t0) * 10
    total = (t["splat_est"] + t["div"] + t["solve"] + t["iso_mc"] + t["sdf_est"] + t["adj_solve"]
             + t["splat_adjoint_est"] + t["query_est"])
    extra = {"triangles": int(mesh["verts"].shape[0]), "sample_lin": lin, "sample_phi": phi_s}
    if count_nodes:
        k = min(count_nodes, node_sample)
        nodes = OP.node_xyz(lin[:k], RES, lo, h)
        cnt = box_candidates(nodes, mesh["verts"], dist[:k])
        extra["alg_tests_per_node"] = float(cnt.mean())
        extra["alg_count_nodes"] = k
    return total, t, extra


def cpu_baseline(node_sample: int):
    p, n, q, g = workload()
    rng = np.random.default_rng(7)
    total, t, extra = oracle_step(p, n, q, g, node_sample, rng, count_nodes=500)
    return {"value": RES ** 3 / total, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 numpy oracle (one thread) on the same step: splat, divergence, DCT solve, "
                       f"iso-value, marching cubes, adjoint solve and splat adjoint on the full 256^3 "
                       f"problem; exact distance on {node_sample} random nodes scaled to all 16.8M; "
                       f"query interpolation on 100k of the 1M points scaled; est. step {total:.1f} s"),
            "stage_s": t, "alg_tests_per_node": extra["alg_tests_per_node"],
            "alg_count_nodes": extra["alg_count_nodes"],
            "_sample": (extra["sample_lin"], extra["sample_phi"])}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    p, n, q, g = workload()
    rng = np.random.default_rng(11)
    times = []
    nodes = min(args.cpu_sample_nodes, 300)
    for k in range(args.warmup + args.steps):
        total, t, _ = oracle_step(p, n, q, g, nodes, rng, point_frac=0.1)
        if k >= args.warmup:
            times.append(total)
    ms = 1e3 * float(np.mean(times))
    value = RES ** 3 / (ms / 1e3)
    cores = 1
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "SH body (degree<=8) 200k points, 256^3 grid, 1M queries, "
                                  "forward + query + adjoint", "res": RES, "points": NPTS, "queries": NQ},
           "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                            "sample": f"per step (FP64 numpy, one thread): divergence, DCT solves, "
                                      f"iso-value and marching cubes on the full 256^3 grid; splat and "
                                      f"splat adjoint on 10% of the points, exact distance on {nodes} "
                                      f"nodes and query on 10% of the queries, each scaled to the full "
                                      f"step"},
           "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--stage-steps", type=int, default=5)
    ap.add_argument("--cpu-sample-nodes", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=300)
    ap.add_argument("--pca-reps", type=int, default=10)
    # smaller cases of the same workload, for profiler captures only (the
    # benchmark figure is the default 256^3 / 200k / 1M configuration)
    ap.add_argument("--res", type=int, default=256)
    ap.add_argument("--points", type=int, default=200_000)
    ap.add_argument("--queries", type=int, default=1_000_000)
    # solver kernels inside graphs with device-side loops cannot be profiled
    # one by one: run the solves as plain launch sequences (profiler only)
    ap.add_argument("--no-graphs", action="store_true")
    args = ap.parse_args()
    globals().update(RES=args.res, NPTS=args.points, NQ=args.queries)
    if args.no_graphs:
        HANDLE_OPTS["use_graphs"] = 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
