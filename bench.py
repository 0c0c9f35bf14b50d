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
    global FP32_PEAK_TFLOPS, FP32_PEAK_KIND
    FP32_PEAK_TFLOPS, FP32_PEAK_KIND = fp32_peak()
    ge.build()
    from paper_2609_20964_gb300 import PREC_FP32, PREC_FP64, Reconstructor

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

    if args.profile:
        # profiler captures: the warm-up and timed steps only, one handle
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "cells/s", "ms_per_step": ms_per_step,
                              "profile_run": True, "timed_stage_ms": timed_stage_ms}))
        rec.close()
        return
    fwd_ms = time_it(lambda: rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf), 5)

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
    oracle_on = rank == 0 and ws == 1 and not args.no_cpu_baseline
    workers = os.cpu_count() or 1
    if oracle_on:
        cpu = cpu_baseline(args.cpu_sample_nodes, workers)
    # mixed precision against plain FP32, each arm checked against the oracle
    prec = None
    if rank == 0 and args.precision_arms:
        oref = oracle_reference(p, n, workers) if oracle_on else None
        prec = precision_arms(Reconstructor, PREC_FP32, PREC_FP64, P, Nn, Q, G, sdf_buf, nrm_buf, oref,
                              args.pca_reps)
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
                   "queries": NQ, "precision": "mixed: float-float iterative refinement (FP64 norms and sums) "
                                                        "around one FP32 spectral (DCT) correction per step "
                                                        "(256 is a power of two)",
                   "l2": "working set > 1 GB per step (fields of 67 MB) exceeds the 129 MB L2; no flush",
                   "parallelism": f"replicas x{ws}",
                   "override": (RES, NPTS, NQ) != (256, 200_000, 1_000_000) or bool(HANDLE_OPTS)},
        "latency_ms": {"p50": statistics.median(step_ms), "p99": float(np.percentile(step_ms, 99))},
        "fwd_cells_per_s": N / (fwd_ms / 1e3),
        "fwd_ms": fwd_ms,
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
    if prec is not None:
        out["precision_arms"] = prec
        best = prec["summary"]["fastest_plain_arm"]
        if best is not None:
            out["fp32_plain_fwd_cells_per_s"] = prec[best]["fwd_cells_per_s"]
            out["fp32_plain"] = {"arm": best, "fwd_ms": prec[best]["fwd_ms"],
                                 "time_to_1e-4_ms": prec[best]["time_to_1e-4_ms"]}
    if rank == 0 and args.wave_steps > 0:
        out["moving_boundary"] = moving_boundary_bench(Reconstructor, args.wave_steps, oracle_on, workers)
    if rank == 0 and ws == 1 and args.serving_requests > 0:
        out["serving"] = serving_bench(args.serving_requests, args.serving_sweep_requests)
    if rank == 0 and args.pca_reps > 0:
        rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf)
        out["galerkin_q1"] = galerkin_q1_bench(Reconstructor, P, Nn, Q, G, sdf_buf.clone(), args.pca_reps)
        out["exact_query"] = exact_query_bench(rec, P, Nn, Q, args.pca_reps)
        out["normal_estimation"] = normal_estimation_bench(rec, P, args.pca_reps, cpu is not None)
        out["normal_orientation"] = orientation_bench(rec, P, n, args.pca_reps)
    if cpu is not None:
        # SDF error of the benchmark handle against the oracle's exact distance on its sampled nodes
        lin, ophi = cpu.pop("_sample")
        rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf)
        idx = torch.from_numpy(lin.astype(np.int64)).cuda()
        extent = float(np.max(BBOX[3:] - BBOX[:3]))
        got = sdf_buf.reshape(-1)[idx].double().cpu().numpy()
        out["sdf_err_vs_oracle"] = {"max_abs_over_extent": float(np.abs(got - ophi).max() / extent),
                                    "nodes": int(len(lin)), "bound": 1e-4}
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

def fp32_peak():
    """FP32 ALU peak of the device: its SM count (device attribute) x 128 FP32
    lanes per SM x 2 flop per FMA x its maximum SM clock (the measured peaks
    file, else nvidia-smi, else 2070 MHz).  Returns (TFLOP/s, description)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz, src = None, None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz, src = float(json.load(f)["sm_max_mhz"]), "measured peaks file"
    except (OSError, KeyError, ValueError):
        pass
    if mhz is None:
        try:
            r = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()),
                                "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                               capture_output=True, text=True, timeout=10)
            mhz, src = float(r.stdout.strip().splitlines()[0]), "nvidia-smi clocks.max.sm"
        except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
            mhz, src = 2070.0, "nominal"
    return sms * 128 * 2 * mhz * 1e6 / 1e12, (f"derived: {sms} SMs (device attribute) x 128 FP32 lanes x "
                                              f"2 flop x {mhz:.0f} MHz ({src})")


FP32_PEAK_TFLOPS = None   # set by fp32_peak() once a device is current
FP32_PEAK_KIND = None
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
                "peak_kind": FP32_PEAK_KIND,
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


# --------------------------------------------------------------- precision arms
PREC_SAMPLE_NODES = 2000       # nodes where the SDF is compared with the oracle
PREC_NORMAL_NODES = 150        # nodes where the normals are compared
PREC_GRAD_QUERIES = 2000       # query seeds of the gradient comparison


def oracle_reference(p, n, workers: int):
    """The oracle's values that every precision arm is checked against, on the
    benchmark body: phi on sampled nodes, stencil normals on sampled nodes, and
    the adjoint (d_points, d_normals) of seeds at sampled queries, with the
    oracle's exact distance evaluated only at the nodes these need."""
    import synth
    from oracle import pipeline as OP
    t0 = time.perf_counter()
    ref = OP.forward_to_mesh(p, n, BBOX, RES)
    rng = np.random.default_rng(17)
    lin_sdf = rng.choice(RES ** 3, PREC_SAMPLE_NODES, replace=False)
    lin_nrm = rng.choice(RES ** 3, PREC_NORMAL_NODES, replace=False)
    qg = synth.uniform_queries(PREC_GRAD_QUERIES, seed=2101)
    g = np.random.default_rng(78).standard_normal(PREC_GRAD_QUERIES).astype(np.float32)
    corners = OP.query_corner_nodes(qg, RES, ref.lo, ref.h)
    OP.fill_nodes(ref, np.concatenate([lin_sdf, corners]), workers)
    phi_sdf = ref.phi.reshape(-1)[lin_sdf].copy()
    nrm, gmag = OP.normals_at(ref, lin_nrm)
    dp, dn, _ = OP.backward(ref, q=qg, d_sdf_q=g.astype(np.float64))
    return {"lin_sdf": lin_sdf, "phi_sdf": phi_sdf, "lin_nrm": lin_nrm, "nrm": nrm, "gmag": gmag,
            "q": qg, "g": g, "dp": dp, "dn": dn, "seconds": time.perf_counter() - t0, "workers": workers}


def _angle_deg(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1)))


def arm_errors(rec, P, Nn, oref, sdf_ref=None):
    """SDF, normal and gradient errors of one handle's result against the
    oracle (oref: sampled nodes, normals, gradients), and the SDF's largest
    difference over all nodes from sdf_ref (the mixed arm's field, itself
    within ~5e-8 of the extent of the oracle's on the sampled nodes)."""
    import torch
    sdf, nrm = rec.reconstruct(P, Nn, BBOX, RES)
    extent = float(np.max(BBOX[3:] - BBOX[:3]))
    info = rec.info()
    out = {"sdf_max_abs_diff_vs_mixed_all_nodes": (float((sdf - sdf_ref).abs().max()) / extent
                                                    if sdf_ref is not None else 0.0),
           "solver_steps": info["solver_steps"], "residual_rel": info["residual_rel"], "status": info["status"]}
    if sdf_ref is None:
        out["sdf"] = sdf.clone()
    if oref is None:
        return out
    lin = torch.from_numpy(oref["lin_sdf"].astype(np.int64)).cuda()
    got = sdf.reshape(-1)[lin].double().cpu().numpy()
    out["sdf_max_abs_over_extent"] = float(np.abs(got - oref["phi_sdf"]).max() / extent)
    ln = torch.from_numpy(oref["lin_nrm"].astype(np.int64)).cuda()
    gn = nrm.reshape(3, -1)[:, ln].T.double().cpu().numpy()
    ok = oref["gmag"] >= 0.9
    out["normal_max_angle_deg"] = float(_angle_deg(gn[ok], oref["nrm"][ok]).max())
    if rec.opt.keep_for_backward:
        Q = torch.from_numpy(oref["q"]).cuda()
        G = torch.from_numpy(oref["g"]).cuda()
        dp, dn, _ = rec.backward(q=Q, d_sdf_q=G)
        for nm, got_t, want in (("d_points", dp, oref["dp"]), ("d_normals", dn, oref["dn"])):
            got = got_t.double().cpu().numpy()
            out[nm + "_rel_err"] = float(np.linalg.norm(got - want) / np.linalg.norm(want))
            out[nm + "_max_point_err"] = float(np.linalg.norm(got - want, axis=1).max()
                                               / np.linalg.norm(want, axis=1).max())
    return out


def arm_times(rec, P, Nn, Q, G, sdf_buf, nrm_buf, reps: int):
    """Median forward (SDF + normals) and forward + query + adjoint times."""
    import torch
    stream = torch.cuda.current_stream()

    def fwd():
        rec.reconstruct(P, Nn, BBOX, RES, sdf_out=sdf_buf, nrm_out=nrm_buf)

    def step():
        fwd()
        rec.query(Q, with_normals=False)
        rec.backward(q=Q, d_sdf_q=G)

    out = {}
    fns = [("fwd_ms", fwd)] + ([("fwd_query_adjoint_ms", step)] if rec.opt.keep_for_backward else [])
    if rec.opt.stage_timing:
        for _ in range(2):
            fwd()
        torch.cuda.synchronize()
        rec.stage_times(reset=True)
        for _ in range(reps):
            fwd()
        torch.cuda.synchronize()
        st = rec.stage_times(reset=True)
        out["solve_ms"] = st["solve"][0] / max(st["solve"][1], 1)
    for name, fn in fns:
        for _ in range(2):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        out[name] = statistics.median(a.elapsed_time(b) for a, b in ev)
    return out


def precision_arms(Reconstructor, PREC_FP32, PREC_FP64, P, Nn, Q, G, sdf_buf, nrm_buf, oref, reps: int):
    """The mixed-precision path against plain FP32 on the same input, each
    timed and checked against the oracle (SDF, normals, gradients):
      mixed            float-float refinement around the spectral correction
                       (the benchmark's configuration);
      mixed_multigrid  the same refinement around FP32 multigrid V-cycles;
      fp64_refinement  the refinement with a native FP64 iterate and residual
                       (the FP64 pipe) instead of float-float;
      fp32_spectral    one direct FP32 spectral solve, no refinement;
      fp32_multigrid   plain FP32 V-cycles, the fewest that bring the SDF
                       within 1e-4 of the extent (a sweep decides).
    The adjoint solve refines in float-float in every arm; the FP32 arms differ
    in their forward state only.  An arm reaches 1e-4 when its SDF lies within
    1e-4 of the extent of the mixed arm's at every node and of the oracle's on
    the sampled nodes; time_to_1e-4 is then its forward time, else null."""
    arms = {}
    specs = [("mixed", {}), ("mixed_multigrid", {"spectral": 0}), ("fp64_refinement", {"precision": PREC_FP64}),
             ("fp32_spectral", {"precision": PREC_FP32, "max_vcycles": 1, "tol_rel": 1e-5})]
    rec = Reconstructor(RES, NPTS, keep_for_backward=0, **HANDLE_OPTS)
    sdf_ref = arm_errors(rec, P, Nn, None)["sdf"]
    rec.close()

    def reaches(e):
        return (e["sdf_max_abs_diff_vs_mixed_all_nodes"] <= 1e-4
                and e.get("sdf_max_abs_over_extent", 0.0) <= 1e-4)

    # the plain multigrid sweep: fewest V-cycles to 1e-4 of the extent
    sweep = []
    best_k = None
    for k in (2, 3, 4, 5, 6, 7, 8, 10, 12, 16):
        rec = Reconstructor(RES, NPTS, precision=PREC_FP32, spectral=0, max_vcycles=k, tol_rel=1e-7,
                            keep_for_backward=0, **HANDLE_OPTS)
        e = arm_errors(rec, P, Nn, oref, sdf_ref)
        rec.close()
        sweep.append({"vcycles": k, "sdf_max_abs_diff_vs_mixed_all_nodes": e["sdf_max_abs_diff_vs_mixed_all_nodes"],
                      "sdf_max_abs_over_extent": e.get("sdf_max_abs_over_extent"),
                      "normal_max_angle_deg": e.get("normal_max_angle_deg"), "residual_rel": e["residual_rel"]})
        if reaches(e):
            best_k = k
            break
    if best_k is not None:
        specs.append(("fp32_multigrid", {"precision": PREC_FP32, "spectral": 0, "max_vcycles": best_k,
                                         "tol_rel": 1e-7}))
    for name, opts in specs:
        rec = Reconstructor(RES, NPTS, stage_timing=1, **opts, **HANDLE_OPTS)
        a = arm_errors(rec, P, Nn, oref, sdf_ref)
        a.pop("sdf", None)
        a.update(arm_times(rec, P, Nn, Q, G, sdf_buf, nrm_buf, reps))
        a["fwd_cells_per_s"] = RES ** 3 / (a["fwd_ms"] / 1e3)
        a["time_to_1e-4_ms"] = a["fwd_ms"] if reaches(a) else None
        a["options"] = {k: v for k, v in opts.items()}
        arms[name] = a
        rec.close()
    arms["fp32_multigrid_sweep"] = sweep
    plain = [(arms[k]["time_to_1e-4_ms"], k) for k in ("fp32_spectral", "fp32_multigrid")
             if k in arms and arms[k]["time_to_1e-4_ms"] is not None]
    tm = arms["mixed"]["time_to_1e-4_ms"]
    arms["summary"] = {
        "mixed_time_to_1e-4_ms": tm,
        "fastest_plain_arm": min(plain)[1] if plain else None,
        "fastest_plain_time_to_1e-4_ms": min(plain)[0] if plain else None,
        "plain_over_mixed_time": (min(plain)[0] / tm) if (plain and tm) else None,
        "errors_against": ("oracle (sampled nodes, normals, gradients) and the mixed arm (all nodes)"
                           if oref is not None else "the mixed arm (all nodes)"),
        "oracle_nodes": PREC_SAMPLE_NODES, "oracle_normal_nodes": PREC_NORMAL_NODES,
        "gradient_seeds": PREC_GRAD_QUERIES,
        "oracle_seconds": oref["seconds"] if oref else None, "oracle_workers": oref["workers"] if oref else None}
    return arms


# ------------------------------------------------------------ moving boundary
WAVE_RES = 192
WAVE_POINTS = 50_000
WAVE_STEPS = 200
WAVE_CHECK = (0, 50, 100, 150, 199)


def moving_boundary_bench(Reconstructor, steps: int, with_oracle: bool, workers: int):
    """The moving-boundary workload (Sec. 3.2: the SDF and normals are
    regenerated at every step): the 0.35/0.08/0.12 ellipsoid bent by the
    travelling lateral wave (reading R14), 50,000 points re-sampled each step,
    192^3 grid (a multigrid solve: 192 is not a power of two), full SDF +
    normal reconstruction per step, mixed precision.  The same series runs
    warm-started (each solve from the previous step's indicator) and cold;
    per-step CUDA-event times on the launching stream, the solver's refinement
    steps, and the SDF error against the oracle at the checked steps (sampled
    nodes)."""
    import torch
    import synth
    stream = torch.cuda.current_stream()
    clouds = [synth.wave_ellipsoid_cloud(t, n=WAVE_POINTS) for t in range(steps)]
    dev = [(torch.from_numpy(p).cuda(), torch.from_numpy(n).cuda()) for p, n in clouds]
    sdf = torch.empty((WAVE_RES,) * 3, device="cuda")
    nrm = torch.empty((3,) + (WAVE_RES,) * 3, device="cuda")
    out = {"res": WAVE_RES, "points": WAVE_POINTS, "steps": steps}
    kept = {}
    # warm-up shape: a sphere sampled like the series (workspaces touched,
    # solver graph recorded); the series' first solve starts from its indicator
    wp, wn = synth.sphere_cloud(WAVE_POINTS, seed=77)
    WP, WN = torch.from_numpy(wp).cuda(), torch.from_numpy(wn).cuda()
    for name, warm in (("warm", 1), ("cold", 0)):
        iters = []
        for timed in (True, False):
            rec = Reconstructor(WAVE_RES, WAVE_POINTS, warm_start=warm, keep_for_backward=0, **HANDLE_OPTS)
            for _ in range(3):
                rec.reconstruct(WP, WN, BBOX, WAVE_RES, sdf_out=sdf, nrm_out=nrm)
            torch.cuda.synchronize()
            if not timed:
                # refinement steps per step, read after each step (reading the
                # handle's info synchronises: kept out of the timed series)
                for P, N in dev:
                    rec.reconstruct(P, N, BBOX, WAVE_RES, sdf_out=sdf, nrm_out=nrm)
                    iters.append(rec.info()["solver_steps"])
                rec.close()
                continue
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for t, (P, N) in enumerate(dev):
                ev[t][0].record(stream)
                rec.reconstruct(P, N, BBOX, WAVE_RES, sdf_out=sdf, nrm_out=nrm)
                ev[t][1].record(stream)
                if t in WAVE_CHECK:
                    kept[(name, t)] = sdf.clone()
            t1.record(stream)
            torch.cuda.synchronize()
            status = rec.info()["status"]
            rec.close()
        ms = [a.elapsed_time(b) for a, b in ev]
        out[name] = {"total_ms": t0.elapsed_time(t1), "ms_per_step_median": statistics.median(ms),
                     "status_last": status,
                     "ms_per_step_mean": float(np.mean(ms)), "ms_per_step_p99": float(np.percentile(ms, 99)),
                     "solver_steps_mean": float(np.mean(iters)), "solver_steps_first": iters[0],
                     "solver_steps_max": int(max(iters)),
                     "cells_per_s": WAVE_RES ** 3 * steps / (t0.elapsed_time(t1) / 1e3)}
    out["warm_max_abs_sdf_diff_vs_cold"] = max(
        float((kept[("warm", t)] - kept[("cold", t)]).abs().max()) for t in WAVE_CHECK if t < steps)
    if with_oracle:
        from oracle import pipeline as OP
        extent = float(np.max(BBOX[3:] - BBOX[:3]))
        errs = {}
        rng = np.random.default_rng(23)
        for t in WAVE_CHECK:
            if t >= steps:
                continue
            p, n = clouds[t]
            ref = OP.forward_to_mesh(p, n, BBOX, WAVE_RES)
            lin = rng.choice(WAVE_RES ** 3, 1000, replace=False)
            ophi, _, _ = OP.sdf_at_pool(ref, lin, workers)
            got = kept[("warm", t)].reshape(-1)[torch.from_numpy(lin).cuda()].double().cpu().numpy()
            errs[str(t)] = float(np.abs(got - ophi).max() / extent)
        out["warm_sdf_err_vs_oracle"] = {"max_abs_over_extent": errs, "nodes_per_step": 1000, "bound": 1e-4}
    return out


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
                        "peak_kind": FP32_PEAK_KIND}}
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
SERVE_QUERIES = 50_000          # query points per request
SERVE_DIR_POOL = 500_000        # seeded unit directions the bodies are sampled at


def serving_inputs(mix):
    """Per request its own random degree-8 SH body (coefficients N(0, 0.02^2)
    fitted into r in [0.1, 0.45]), sampled on the device by the library's
    generator (wgeo_sh_surface) at n_i seeded uniform directions (a window of
    a device-resident pool), 50,000 uniform queries drawn on the device, and
    for the gradient requests a seeded adjoint seed at the queries.  All
    device-resident before the arrivals start."""
    import torch
    import synth
    from paper_2609_20964_gb300 import sh_surface
    pool = torch.from_numpy(synth.uniform_dirs(SERVE_DIR_POOL, np.random.default_rng(50_001))
                            .astype(np.float32)).cuda()
    gen = torch.Generator(device="cuda")
    out = []
    for r in mix:
        rng = np.random.default_rng(r["seed"])
        theta = torch.from_numpy(synth.random_sh_body_theta(8, rng).astype(np.float32)).cuda()
        n = min(r["n"], SERVE_DIR_POOL)
        off = int(rng.integers(0, SERVE_DIR_POOL - n + 1))
        P, N = sh_surface(theta, pool[off:off + n])
        gen.manual_seed(r["seed"])
        Q = torch.rand((SERVE_QUERIES, 3), generator=gen, device="cuda")
        G = (torch.randn(SERVE_QUERIES, generator=gen, device="cuda") / SERVE_QUERIES) if r["grad"] else None
        out.append((r, P, N, Q, G))
    torch.cuda.synchronize()
    return out


def _serve(srv, reqs, rate, Request):
    """Submits `reqs` at their exponential gaps scaled to `rate` (requests per
    second); returns (results, wall seconds, queue depths seen at each arrival)."""
    depth, futs = [], []
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
    return results, time.perf_counter() - t0, depth


def serving_bench(n_req: int, sweep_req: int, loads=(0.8, 0.5, 1.0, 1.2), streams: int = 4):
    """The serving workload: requests with grid sizes {64, 128, 256}^3 w.p.
    {0.5, 0.35, 0.15}, point counts log-uniform in [1e4, 5e5], half of them
    with the adjoint of a loss at their queries, Poisson arrivals (reading
    R15) at offered loads rho of the measured serial capacity, through the
    request loop (continuous batching on `streams` streams, HBM-budget
    admission, handles pooled per grid size and point-count bucket, warm
    start on).  Latency = completion - scheduled arrival, queueing included.
    The first load runs `n_req` requests, the others `sweep_req`."""
    import torch
    import synth
    from paper_2609_20964_gb300.serving import Request, Server
    mix = synth.serving_requests(n_req)
    reqs = serving_inputs(mix)
    srv = Server(budget_bytes=48 << 30, n_streams=streams, max_points=500_000)
    # serial capacity: a sample of the mix one at a time (also creates the
    # pooled workspaces and records the solver graphs)
    sample = reqs[: min(96, len(reqs))]
    for r, P, N, Q, G in sample[:24]:
        srv.submit(Request(points=P, normals=N, res=r["res"], queries=Q, d_sdf_q=G)).result()
    t0 = time.perf_counter()
    for r, P, N, Q, G in sample:
        srv.submit(Request(points=P, normals=N, res=r["res"], queries=Q, d_sdf_q=G)).result()
    serial_s = (time.perf_counter() - t0) / len(sample)
    out = {"requests": n_req, "streams": streams, "serial_service_ms": 1e3 * serial_s,
           "queries_per_request": SERVE_QUERIES, "with_gradients": int(sum(r["grad"] for r in mix)),
           "bodies": "one random degree-8 SH body per request, sampled on the device by wgeo_sh_surface",
           "point_buckets": list(srv.buckets), "warm_start": 1,
           "order": f"fewest grid cells first; the oldest once it has waited {1e3 * srv.max_wait_s:.0f} ms",
           "loads": {}}
    for k, rho in enumerate(loads):
        sub = reqs if k == 0 else reqs[:sweep_req]
        srv.latencies.clear()
        srv.latencies_by_res.clear()
        rate = rho / serial_s
        results, wall, depth = _serve(srv, sub, rate, Request)
        st = srv.stats()
        lat = np.array([x.latency_s for x in results]) * 1e3
        cells = sum(r["res"] ** 3 for r, *_ in sub)
        points = sum(min(r["n"], SERVE_DIR_POOL) for r, *_ in sub)
        out["loads"][str(rho)] = {
            "requests": len(sub), "offered_rate_per_s": rate,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "cells_per_s": cells / wall, "points_per_s": points / wall,
            "wall_s": wall, "queue_depth_max": int(max(depth)), "queue_depth_mean": float(np.mean(depth)),
            "by_res": {str(r): v for r, v in st["by_res"].items()},
            "status_nonzero": int(sum(1 for x in results if x.info["status"] != 0))}
    out["used_bytes"] = srv.used_bytes
    srv.close()
    first = out["loads"][str(loads[0])]
    out.update({"offered_load": loads[0], "p50_ms": first["p50_ms"], "p99_ms": first["p99_ms"],
                "cells_per_s": first["cells_per_s"]})
    return out


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


def oracle_step(p, n, q, g, node_sample: int, rng, count_nodes: int = 0, pool=None):
    """One step of the oracle on the benchmark workload: every stage on the
    full problem except the exact distance + sign, which runs on `node_sample`
    random nodes (on `pool` when given) and is scaled to all nodes, and the
    query interpolation, run on a tenth of the queries and scaled.  Returns
    (estimated seconds for the full step, per-stage seconds, detail dict).
    The same sampling serves the CPU baseline and the reference arm; with
    `pool` (started and warmed beforehand) the distance sample runs on it."""
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
    t0 = time.perf_counter()
    bins, fin, _ = OG.bin_points(pp, BBOX, RES)
    V = OS.splat(pp, nn, bins, fin, lo, h, RES)
    t["splat"] = time.perf_counter() - t0
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
    phi_s, dist, _ = OP.sdf_at_pool(rec, lin, pool=pool)
    t["sdf_sample"] = time.perf_counter() - t0
    t["sdf_est"] = t["sdf_sample"] * N / node_sample
    # stencil normals cost ~ one more distance per node in the oracle's own form: counted as 0
    # adjoint: the adjoint solve (the same operator and cost as the forward's) and the splat adjoint
    t0 = time.perf_counter()
    lam = OPo.solve(chi)
    t["adj_solve"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    dV = D.divergence_adjoint(lam)
    OS.splat_adjoint(pp, nn, bins, fin, lo, h, RES, dV)
    t["splat_adjoint"] = time.perf_counter() - t0
    # trilinear query at the 1M points (vectorised, measured on a tenth, scaled)
    qs = q[: len(q) // 10].astype(np.float64)
    t0 = time.perf_counter()
    OI.trilinear(qs, lo, h, RES)
    t["query_est"] = (time.perf_counter() - t0) * 10
    total = (t["splat"] + t["div"] + t["solve"] + t["iso_mc"] + t["sdf_est"] + t["adj_solve"]
             + t["splat_adjoint"] + t["query_est"])
    extra = {"triangles": int(mesh["verts"].shape[0]), "sample_lin": lin, "sample_phi": phi_s}
    if count_nodes:
        k = min(count_nodes, node_sample)
        nodes = OP.node_xyz(lin[:k], RES, lo, h)
        cnt = box_candidates(nodes, mesh["verts"], dist[:k])
        extra["alg_tests_per_node"] = float(cnt.mean())
        extra["alg_count_nodes"] = k
    return total, t, extra


ORACLE_SAMPLE = ("FP64 numpy oracle on the benchmark step: binning, splat, divergence, DCT solve, iso-value, "
                 "marching cubes, adjoint solve and splat adjoint on the full 256^3 problem and all 200k points; "
                 "exact distance + sign on {nodes} random nodes scaled to all 16.8M; query interpolation on "
                 "100k of the 1M queries scaled")


def c1_full_step(workers: int):
    """One oracle step on the 4,096-point sphere at 64^3, end to end and
    unscaled: the whole forward on every node (exact distance by `workers`
    processes), query at 100k points and the adjoint of a loss on them."""
    import synth
    from oracle import pipeline as OP
    ci = synth.config_inputs("sphere64")
    q = ci["queries"]
    g = np.random.default_rng(1).standard_normal(len(q)) / len(q)
    t0 = time.perf_counter()
    rec = OP.reconstruct(ci["points"], ci["normals"], ci["bbox"], ci["res"], workers=workers)
    OP.query(rec, q)
    OP.backward(rec, q=q, d_sdf_q=g)
    sec = time.perf_counter() - t0
    return {"value": ci["res"] ** 3 / sec, "unit": "cells/s", "seconds": sec, "cores": workers,
            "workload": "sphere r=0.3, 4,096 points, 64^3, 100k queries: forward on every node, query, "
                        "adjoint; nothing sampled or scaled"}


def cpu_baseline(node_sample: int, workers: int):
    p, n, q, g = workload()
    total, t, extra = oracle_step(p, n, q, g, node_sample, np.random.default_rng(7), count_nodes=500)
    out = {"value": RES ** 3 / total, "unit": "cells/s", "cores": 1, "kind": "oracle",
           "sample": ORACLE_SAMPLE.format(nodes=node_sample) + f"; one thread; est. step {total:.1f} s",
           "stage_s": t, "alg_tests_per_node": extra["alg_tests_per_node"],
           "alg_count_nodes": extra["alg_count_nodes"],
           "_sample": (extra["sample_lin"], extra["sample_phi"])}
    if workers > 1:
        # the same step with a larger distance sample on every host core (the
        # other stages are single numpy calls), on a pool started and warmed
        # first so that its start-up is not timed
        import multiprocessing as mp
        from oracle import sdf as OS
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(OS._exact_distance_part, [(np.zeros((1, 3)), np.zeros((1, 3, 3)))] * workers)
            tot_all, t_all, _ = oracle_step(p, n, q, g, 8 * node_sample, np.random.default_rng(8), pool=pool)
        out["all_cores"] = {"value": RES ** 3 / tot_all, "unit": "cells/s", "cores": workers,
                            "est_step_s": tot_all, "sdf_sample_nodes": 8 * node_sample,
                            "sdf_sample_s": t_all["sdf_sample"]}
        out["c1_full_step"] = c1_full_step(workers)
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    p, n, q, g = workload()
    rng = np.random.default_rng(11)
    times = []
    for k in range(args.warmup + args.steps):
        total, t, _ = oracle_step(p, n, q, g, args.cpu_sample_nodes, rng)
        if k >= args.warmup:
            times.append(total)
    ms = 1e3 * float(np.mean(times))
    value = RES ** 3 / (ms / 1e3)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "SH body (degree<=8) 200k points, 256^3 grid, 1M queries, "
                                  "forward + query + adjoint", "res": RES, "points": NPTS, "queries": NQ,
                      "precision": "f64 oracle"},
           "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                            "sample": ORACLE_SAMPLE.format(nodes=args.cpu_sample_nodes) + "; one thread; "
                                      "each step scaled to the full step as the CPU baseline is"},
           "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--stage-steps", type=int, default=5)
    ap.add_argument("--cpu-sample-nodes", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--serving-sweep-requests", type=int, default=500)
    ap.add_argument("--pca-reps", type=int, default=10)
    # mixed precision against plain FP32 (each arm timed and checked against the oracle)
    ap.add_argument("--precision-arms", type=int, default=1)
    # the moving-boundary series (192^3 wave ellipsoid), steps; 0 skips it
    ap.add_argument("--wave-steps", type=int, default=200)
    # smaller cases of the same workload, for profiler captures only (the
    # benchmark figure is the default 256^3 / 200k / 1M configuration)
    ap.add_argument("--res", type=int, default=256)
    ap.add_argument("--points", type=int, default=200_000)
    ap.add_argument("--queries", type=int, default=1_000_000)
    # solver kernels inside graphs with device-side loops cannot be profiled
    # one by one: run the solves as plain launch sequences (profiler only)
    ap.add_argument("--no-graphs", action="store_true")
    # profiler captures: only the warm-up and timed steps of the main handle,
    # optionally with another solve precision
    ap.add_argument("--profile", action="store_true")
    ap.add_argument("--precision", choices=["mixed", "fp32", "fp64"], default="mixed")
    args = ap.parse_args()
    globals().update(RES=args.res, NPTS=args.points, NQ=args.queries)
    if args.no_graphs:
        HANDLE_OPTS["use_graphs"] = 0
    if args.precision != "mixed":
        if not args.profile:
            raise SystemExit("--precision applies to --profile runs only")
        HANDLE_OPTS["precision"] = {"fp32": 1, "fp64": 2}[args.precision]
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
