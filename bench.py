#!/usr/bin/env python3
"""Benchmark of the GB300 DW-FMM matvec (one JSON line on rank 0).

A step is one DW-FMM matvec y = K_tilde x (gather, P2M, M2M, M2L, L2L, L2P,
P2P, scatter) over one batch of R right-hand sides on a resident tree; the
expansion setup (weights, index set, nodes, V^{-1}) and the tree build
(tree, lists, cluster data) are timed separately and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the float64 CPU oracle on the same workload (a
bounded sample per step: the rows of one target leaf per host core, each
core with its own full upward pass).  Under torchrun each rank runs an independent replica (the method
runs on one GPU; replicas scale weakly); rank 0 prints.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DW-FMM matvec pts·RHS/s and CG solve p50/p99 ms, mixed vs FP64 @ rel err 1e-6"
UNIT = "pts·RHS/s"
FP32_LANES = 128


def workload(name: str):
    import dwfmm_inputs as di
    table = {"mixed": di.mixed_gauss_d10, "fp64": di.fp64_matern_d8, "small": di.small_exp_d4}
    return table[name]()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle sample (its own process, no GPU; one worker per host core)
# ---------------------------------------------------------------------------

def _oracle_leaves(pb, count):
    """`count` target leaves spread evenly over the tree order."""
    first = (1 << pb.tree.depth) - 1
    nleaf = 1 << pb.tree.depth
    return [first + (i * nleaf) // count for i in range(count)]


def _ancestors(leaf):
    anc, c = [], leaf
    while True:
        anc.append(c)
        if c == 0:
            return anc
        c = (c - 1) // 2


def _oracle_worker(pb, f, leaf, steps, warmup, barrier, out):
    """One host core: the far-field coefficients of the leaf's ancestors
    (setup), then warm-up and timed steps of the leaf-restricted matvec.
    Every step starts at a barrier, so the workers' steps overlap."""
    import os as _os
    from oracle import dwfmm_oracle as o
    t0 = time.time()
    anc = set(_ancestors(leaf))
    for lvl in pb.lists.far:
        for (t, s) in lvl:
            if int(t) in anc:
                o.problem_coefficient(pb, int(t), int(s))
    setup = time.time() - t0
    times = []
    for k in range(warmup + steps):
        barrier.wait()
        t = time.perf_counter()
        o.fmm_matvec_leaves(pb, f, [leaf])
        if k >= warmup:
            times.append(time.perf_counter() - t)
    out.put((leaf, setup, times, _os.getpid()))


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(name: str, steps: int, warmup: int, workers: int = 0):
    """Time the float64 oracle's matvec restricted to target leaves, one leaf
    per host core (full upward pass, far field of the leaf's ancestors, near
    field), all cores stepping together.  The problem and the transfer
    matrices are built once before the workers fork (setup, as on the GPU);
    this process never touches a GPU."""
    import multiprocessing as mp
    import numpy as np
    import dwfmm_inputs as di
    from oracle import dwfmm_oracle as o
    w = workload(name)
    X, f = di.sites_and_rhs(w)
    W = workers or (os.cpu_count() or 1)
    t0 = time.time()
    pb = o.make_problem(X, w.kernel, o.weights_inv_gamma(w.gamma), w.q, w.leaf, w.eta, w.sigma)
    for c in range(1, pb.tree.nclusters):
        o.problem_transfer(pb, c)
    setup_s = time.time() - t0
    leaves = _oracle_leaves(pb, W)
    ctx = mp.get_context("fork")
    barrier = ctx.Barrier(len(leaves))
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(pb, f, leaf, steps, warmup, barrier, q)) for leaf in leaves]
    for p in procs:
        p.start()
    res = [q.get() for _ in procs]
    for p in procs:
        p.join()
    step_s = [max(r[2][k] for r in res) for k in range(steps)]   # the slowest core bounds each step
    rows = sum(int(pb.tree.end[leaf] - pb.tree.begin[leaf]) for leaf in leaves)
    return {"units_per_step": rows * w.nrhs, "s_per_step": statistics.mean(step_s), "steps": steps,
            "setup_s": setup_s + max(r[1] for r in res), "rows": rows, "leaves": len(leaves),
            "cores": len(leaves), "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def oracle_sample_text(res, nrhs):
    return (f"float64 numpy oracle, {res['leaves']} target leaves ({res['rows']} rows x {nrhs} RHS) of the "
            f"same workload per step, one leaf per host core, all cores stepping together: each core runs "
            f"the full upward pass, the far field of its leaf's ancestors and the near field; problem, tree, "
            f"lists and transfer matrices built before timing ({res['setup_s']:.0f} s); mean of "
            f"{res['steps']} steps; {res['cores']} of {res['nproc']} cores ({res['cpu_model']})")


def start_oracle_subprocess(name: str, steps: int, warmup: int):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", name, "--steps", str(steps),
           "--warmup", str(warmup)]
    return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)


def finish_oracle_subprocess(p, timeout: float = 600.0):
    try:
        out, err = p.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        p.kill()
        return None
    for line in out.splitlines()[::-1]:
        line = line.strip()
        if line.startswith("{"):
            return json.loads(line)
    return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def max_over_ranks(dist, device, x: float) -> float:
    """The largest value over the ranks (the slowest replica bounds the job);
    x itself on a single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, n: int, nrhs: int, seconds_per_step: float) -> float:
    """Whole-job points x RHS per second: every rank processes its own
    replica of N x R per step, and the step takes the slowest rank's time."""
    return world * n * nrhs / seconds_per_step


def near_pairs(plan):
    """(ordered near pairs of sites, sum over leaves of |leaf|^2): the pairs of
    every near block (T, S) of Eq. (5.1), and the pairs of its diagonal
    blocks (T, T)."""
    import numpy as np
    t = plan.export_tree()
    _, near = plan.export_lists()
    size = (t["end"] - t["begin"]).astype(np.int64)
    diag = near[near[:, 0] == near[:, 1], 0]
    return int(np.sum(size[near[:, 0]] * size[near[:, 1]])), int(np.sum(size[diag] ** 2))


def p2p_accounting(engine: str, pairs: int, diag: int, d: int, R: int):
    """Algorithmic work of one near-field launch per engine: kernel
    evaluations (each 3d + 4 FP32 flops: d differences or products, d
    multiply-adds, ~4 for phi) and where the 2R flops per ordered pair of the
    contraction run.  The symmetric engine evaluates each unordered pair of
    sites once: (pairs + diag) / 2 evaluations."""
    if engine == "mixed_symmetric_fp16_tensor_exponent":
        return {"evals": (pairs + diag) // 2, "flops_per_eval": 3 * d + 4, "tensor": True,
                "source": "p2p_sym.cu",
                "kernel": ("p2p (near field): k_near_sym_gtc, each unordered near pair of sites evaluated once: "
                           "the exponent 2x'.s' (2d flops) and both contractions on tcgen05 FP16 hi/lo, exp2 and "
                           "the FP16 split on the CUDA cores; the 3d + 4 flops of the evaluation are counted "
                           "against the FP32 peak, the tensor-pipe flops beside them")}
    if engine == "mixed_symmetric_fp16_tensor":
        return {"evals": (pairs + diag) // 2, "flops_per_eval": 3 * d + 4, "tensor": True,
                "source": "p2p_sym.cu",
                "kernel": ("p2p (near field): k_near_sym_tc, each unordered near pair of sites evaluated once on "
                           "the FP32 pipe; both contractions (forward and transposed) on tcgen05 FP16 hi/lo, "
                           "counted separately below")}
    if engine == "mixed_tf32_tensor":
        return {"evals": pairs, "flops_per_eval": 3 * d + 4, "tensor": True, "source": "p2p_tc.cu",
                "kernel": ("p2p (near field): k_sum_tc, every ordered pair evaluated on the FP32 pipe, "
                           "contraction on tcgen05 TF32 hi/lo (counted separately below)")}
    return {"evals": pairs, "flops_per_eval": 3 * d + 4 + 2 * R, "tensor": False, "source": "p2p_f32.cu",
            "kernel": "p2p (near field): k_sum_f32, evaluation and contraction on the FP32 pipe"}


def phase_rooflines(iso_ms: dict, N: int, R: int, d: int, n: int, n_far: int, depth: int, evals_p2p: int,
                    fp32_peak: float, hbm_peak: float, far_engine: str = "", tensor_peak: float = 0.0) -> dict:
    """Per-phase algorithmic work over the phase's isolated time, against the
    peak that applies to it.  Models (stated per phase):
      p2p      kernel evaluations x (3d + 4) flops, FP32 peak (contraction on
               the tensor cores, not counted here)
      m2l      n^2 node pairs per far block x (3d + 4) flops, FP32 peak
      p2m_m2m  2 N n R (leaf moments) + (C - 1) 2 n^2 R (transfers to the
               parents) flops, FP32 peak
      l2l_l2p  the same count for the downward pass and the evaluation at the
               sites, FP32 peak
      (far engine "mixed_fp16_tensor": p2m_m2m and l2l_l2p run as FP16 hi/lo
      contractions on the tensor cores, four products per term: 4x those
      flops against the dense FP16 tensor peak, the measured bf16 figure,
      the same nominal rate)
      gather   N R (8 + 4) bytes (float64 in, float32 leaf blocks out), HBM peak
      scatter  N R (2 x 4 + 8) bytes (near and far float32 in, float64 out), HBM peak"""
    C = (1 << (depth + 1)) - 1
    work = {
        "p2p": (evals_p2p * (3 * d + 4), "flop", fp32_peak, "TFLOP/s"),
        "m2l": (n_far * n * n * (3 * d + 4), "flop", fp32_peak, "TFLOP/s"),
        "p2m_m2m": (2 * N * n * R + (C - 1) * 2 * n * n * R, "flop", fp32_peak, "TFLOP/s"),
        "l2l_l2p": (2 * N * n * R + (C - 1) * 2 * n * n * R, "flop", fp32_peak, "TFLOP/s"),
        "gather": (N * R * 12, "byte", hbm_peak, "GB/s"),
        "scatter": (N * R * 16, "byte", hbm_peak, "GB/s"),
    }
    tensor = far_engine == "mixed_fp16_tensor" and tensor_peak > 0
    if tensor:
        for k in ("p2m_m2m", "l2l_l2p"):
            amount = work[k][0]
            work[k] = (4 * amount, "tensor flop", tensor_peak, "TFLOP/s")
    out = {}
    for k, (amount, kind, peak, unit) in work.items():
        ms = iso_ms.get(k)
        if not ms:
            continue
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        achieved = amount / (ms / 1e3) / scale
        out[k] = {"ms": ms, "algorithmic": amount, "kind": kind, "achieved": achieved, "peak": peak,
                  "unit": unit, "frac": achieved / peak}
    if tensor:
        for k in ("p2m_m2m", "l2l_l2p"):
            if k in out:
                out[k]["engine"] = "tcgen05 kind::f16, FP16 hi/lo, 4 products; two launches per tree level"
    return out


def kernel_source_sha(src: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_2402_09531_gb300", "csrc", src), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def _traffic_records():
    """DRAM traffic per launch recorded from ncu captures, one line per
    (kernel source, workload) in the profile summaries:
    `traffic: <bytes> B per launch; source <file> sha16 <hash>; workload <name>`."""
    import re
    out = []
    pdir = os.path.join(ROOT, "profiles")
    pat = re.compile(r"traffic: ([0-9.eE+]+) B per launch; source (\S+) sha16 ([0-9a-f]{16}); workload (\S+)")
    for fn in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not fn.endswith(".md"):
            continue
        with open(os.path.join(pdir, fn)) as fh:
            for m in pat.finditer(fh.read()):
                out.append((float(m.group(1)), m.group(2), m.group(3), m.group(4), fn))
    return out


def recorded_traffic(src: str, workload_name: str):
    """The recorded traffic of this exact kernel source on this workload, else
    None (the counters no longer describe the kernel that ran)."""
    sha = kernel_source_sha(src)
    for b, s_, h, wl, _ in _traffic_records():
        if s_ == src and h == sha and wl == workload_name:
            return b
    return None


def traffic_basis(src: str, workload_name: str):
    sha = kernel_source_sha(src)
    for b, s_, h, wl, fn in _traffic_records():
        if s_ == src and h == sha and wl == workload_name:
            return f"dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu, profiles/{fn})"
    return f"none: no ncu capture of {src} at sha16 {sha} on this workload"


def compare_fp64(plan, w, Xd, xd, yd, stream, ms_mixed):
    """The plain float64 GPU DW-FMM on the same workload (one matvec) beside
    the timed mixed result yd: float64 time, speed-up, and the relative
    difference of yd, worst column and whole block."""
    import torch
    from paper_2402_09531_gb300 import Plan
    p64 = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, q=w.q, eta=w.eta, leaf_size=w.leaf,
               precision="fp64", max_rhs=int(xd.shape[0]))
    p64.tree_build(Xd)
    y64 = torch.empty_like(xd)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    p64.matvec(xd, y64)
    b.record(stream)
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b)
    diff = yd - y64
    col = torch.linalg.norm(diff, dim=1) / torch.linalg.norm(y64, dim=1)
    block = float(torch.linalg.norm(diff) / torch.linalg.norm(y64))
    p64.close()
    return {"fp64_ms_per_step": ms64, "speedup_vs_fp64": ms64 / ms_mixed,
            "rel_diff_vs_fp64_worst_column": float(col.max()), "rel_diff_vs_fp64_block": block,
            "rel_diff_vs_fp64_columns": [float(v) for v in col],
            "note": "the timed mixed result against one float64 matvec of the same plan parameters and "
                    "inputs (first float64 call, workspace allocation included)"}


def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    import dwfmm_inputs as di
    from paper_2402_09531_gb300 import Plan

    w = workload(args.workload)
    if args.n:
        import dwfmm_inputs as di
        w = di.scaled(w, args.n)
    w.seed = w.seed + 1000 * rank          # independent replica per rank
    X, f = di.sites_and_rhs(w)
    N, R, d = w.n, w.nrhs, w.d
    stream = torch.cuda.current_stream(dev)

    t0 = time.perf_counter()
    plan = Plan(d=d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, q=w.q, eta=w.eta,
                leaf_size=w.leaf, precision=args.precision, max_rhs=R)
    plan.set_m2l_engine(args.m2l_engine)
    setup_ms = (time.perf_counter() - t0) * 1e3
    Xd = torch.from_numpy(X).to(dev)
    torch.cuda.synchronize()
    tree_ms = []
    for _ in range(2):
        t0 = time.perf_counter()
        plan.tree_build(Xd)
        torch.cuda.synchronize()
        tree_ms.append((time.perf_counter() - t0) * 1e3)
    n_x, n_far, n_near, depth = plan.info()
    pairs, diag_pairs = near_pairs(plan)

    xd = torch.from_numpy(f).to(dev)
    yd = torch.empty_like(xd)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        plan.matvec(xd, yd)
    torch.cuda.synchronize()

    plan.set_profiling(True)
    plan.phase_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()                      # evict L2 (129 MB) between steps
            ev[k][0].record(stream)
            plan.matvec(xd, yd)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    phases = plan.phase_times(reset=True)
    # per-phase times with every phase alone on the GPU (not part of the value)
    plan.set_profiling(True, serialize=True)
    for _ in range(2):
        plan.matvec(xd, yd)
    iso = plan.phase_times(reset=True)
    plan.set_profiling(False)
    ms = statistics.mean(step_ms)
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(dist, dev, total_ms)
    ms_max = total_ms / args.steps
    value = job_throughput(world, N, R, ms_max / 1e3)

    # e2e through the public API with host buffers (pinned), copies inside
    xh = torch.from_numpy(f).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        plan.matvec(xh, yh)
    e2e_s = []
    with ClockSampler(local) as clk2:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.matvec(xh, yh)               # synchronises (host y)
            e2e_s.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(dist, dev, statistics.mean(e2e_s))

    # roofline of the dominant kernel (P2P): algorithmic FP32 flops per launch
    # (see p2p_accounting); the tensor-pipe flops of the contraction beside it
    p2p_ms, p2p_launches = phases["p2p"]
    p2p_avg_ms = p2p_ms / max(1, p2p_launches)
    engine = plan.near_engine()
    acct = p2p_accounting(engine, pairs, diag_pairs, d, R)
    achieved = acct["evals"] * acct["flops_per_eval"] / (p2p_avg_ms / 1e3) / 1e12
    peaks = measured_peaks()
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES * 2 * clock_mhz * 1e6 / 1e12
    launches = sum(v[1] for k, v in phases.items() if k != "matvec")
    ksrc = acct["source"]
    traffic = recorded_traffic(ksrc, w.name) if args.precision != "fp64" else None

    solve = None
    if not args.no_solve and rank == 0:
        solve = run_solve_sample(args)

    # CPU oracle baseline (its own process, host cores only) runs while the
    # float64 comparison occupies the GPU
    cpu_proc = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_proc = start_oracle_subprocess(args.workload, args.cpu_steps, 1)

    fp64 = None
    if not args.no_fp64 and rank == 0 and args.precision != "fp64":
        fp64 = compare_fp64(plan, w, Xd, xd, yd, stream, ms_max)

    cpu = None
    if cpu_proc is not None:
        res = finish_oracle_subprocess(cpu_proc)
        if res:
            cpu = {"value": res["units_per_step"] / res["s_per_step"], "unit": UNIT, "cores": res["cores"],
                   "kind": "oracle", "sample": oracle_sample_text(res, R)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision != "fp64" else "f64",
            "data": "synthetic (uniform sites in prod_k [-gamma_k, gamma_k], N(0,1) right-hand sides)",
            "config": {"workload": w.name, "d": d, "N": N, "nrhs": R, "kernel": w.kernel, "q": w.q,
                       "weights": "omega_k = gamma_1/gamma_k", "n_x": n_x, "leaf": w.leaf, "eta": w.eta,
                       "depth": depth, "far_blocks": n_far, "near_blocks": n_near, "near_pairs": pairs,
                       "precision": args.precision, "parallelism": f"replicas x{world}",
                       "l2": "flushed between steps (512 MiB write)"},
            "e2e": {"value": job_throughput(world, N, R, e2e_t), "unit": UNIT, "h2d_bytes_per_step": int(xh.numel() * 8),
                    "d2h_bytes_per_step": int(yh.numel() * 8)},
            "gpu_launches": int(launches),
            "roofline": {"kernel": acct["kernel"], "near_engine": engine,
                         "bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                         "flops_per_eval": acct["flops_per_eval"], "evals_per_launch": acct["evals"],
                         "ordered_pairs_per_launch": pairs,
                         "tensor_flops_per_ordered_pair": (3 * 2 * 16) if acct["tensor"] else 0,
                         "tensor_tflops": (pairs * 96 / (p2p_avg_ms / 1e3) / 1e12) if acct["tensor"] else 0.0,
                         "launch_ms": p2p_avg_ms,
                         "traffic_basis": traffic_basis(ksrc, w.name) if args.precision != "fp64" else None,
                         "peak_basis": f"{sms} SMs x {FP32_LANES} FP32 lanes x 2 flop x {clock_mhz:.0f} MHz "
                                       f"(derived: no measured FP32 peak)"},
            "phase_ms_isolated": {k: v[0] / 2 for k, v in iso.items()},
            "far_engine": plan.far_engine(),
            "m2l_engine": plan.m2l_engine(), "m2l_tune_ms": {"symmetric": plan.m2l_tune_ms()[0],
                                                              "ordered": plan.m2l_tune_ms()[1]},
            "phase_roofline": phase_rooflines({k: v[0] / 2 for k, v in iso.items()}, N, R, d, n_x, n_far, depth,
                                              acct["evals"], peak, float(peaks.get("hbm_gbs", 6804.8)),
                                              plan.far_engine(), float(peaks.get("bf16_tflops", 1900.0))),
            "phase_ms_concurrent": {"note": "timed steps; the far-field phases run on the caller's stream "
                                            "while the near field occupies the GPU from a second stream, so "
                                            "their times include waiting for it",
                                    **{k: v[0] / args.steps for k, v in phases.items()}},
            "setup_ms": setup_ms, "tree_build_ms": min(tree_ms),
            "clocks": clk.summary(), "clocks_e2e": clk2.summary(),
            "cpu_baseline": cpu,
            "solve": solve,
            "fp64_comparison": fp64,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def _serve(reqs, precision, lam, batched=False):
    from paper_2402_09531_gb300.serving import Request, Server, summarize
    rs = [Request(rid=r.rid, X=r.X, f=r.f, kernel=r.kernel, gamma=r.gamma, q=r.q, eta=r.eta, leaf=r.leaf,
                  weight_rule=r.weight_rule, lam=lam, rtol=r.rtol, maxit=r.maxit) for r in reqs]
    srv = Server(precision=precision, max_active=8, batched=batched)
    srv.run(rs[:1])                                     # warm-up (plan pool, kernel attributes)
    srv.batch_rebuilds = 0
    t0 = time.perf_counter()
    res = srv.run(rs)
    out = summarize(res, time.perf_counter() - t0)
    out.update({"precision": precision, "lambda": lam, "peak_active": srv.peak_active, "batched": batched})
    if batched:
        out["batch_rebuilds"] = srv.batch_rebuilds
    srv.close()
    return out


def _serve_poisson(reqs, precision, lam, loads=(0.5, 0.8, 1.0), seed=7, batched=False):
    """Offered-load sweep: the closed-loop rate (all requests at t=0) sets the
    scale; then Poisson arrivals at each fraction of it (seeded exponential
    gaps), p50/p99 latency measured from each request's arrival."""
    import numpy as np
    from paper_2402_09531_gb300.serving import Request, Server, summarize
    base = _serve(reqs, precision, lam, batched=batched)
    rate = base["solves_per_s"]
    rng = np.random.default_rng(seed)
    out = {"closed_loop_solves_per_s": rate, "requests": len(reqs)}
    for load in loads:
        gaps = rng.exponential(1.0 / (load * rate), size=len(reqs))
        arrival = np.cumsum(gaps) - gaps[0]
        rs = [Request(rid=r.rid, X=r.X, f=r.f, kernel=r.kernel, gamma=r.gamma, q=r.q, eta=r.eta, leaf=r.leaf,
                      weight_rule=r.weight_rule, lam=lam, rtol=r.rtol, maxit=r.maxit, arrival=float(a))
              for r, a in zip(reqs, arrival)]
        srv = Server(precision=precision, max_active=8, batched=batched)
        srv.run([dataclasses.replace(rs[0], rid=-1, arrival=0.0)])   # warm-up (plan pool)
        t0 = time.perf_counter()
        res = srv.run(rs)
        summ = summarize(res, time.perf_counter() - t0)
        out[f"load_{load:g}"] = {"offered_per_s": load * rate, **{k: summ[k] for k in
                                 ("ok", "p50_ms", "p99_ms", "solves_per_s", "mean_iters")},
                                 "peak_active": srv.peak_active}
        srv.close()
    return out


def _sample_requests(count, nmax, nmin=0):
    """The first `count` requests of the serving stream with nmin <= N <= nmax
    (eta=2, Sec. 6.2 weights: the readings for the stream's unstated
    parameters)."""
    import dwfmm_inputs as di
    from paper_2402_09531_gb300.serving import Request
    reqs = []
    for w in di.serving_requests(2000):
        if w.n > nmax or w.n < nmin:
            continue
        X, f = di.sites_and_rhs(w, nrhs=1)
        reqs.append(Request(rid=len(reqs), X=X, f=f, kernel=w.kernel, gamma=w.gamma, q=w.q, eta=2.0,
                            leaf=w.leaf, weight_rule="paper_logrho", lam=w.lam, rtol=w.rtol, maxit=4000))
        if len(reqs) >= count:
            break
    return reqs


def run_solve_sample(args):
    """CG solve latency on a bounded sample of the serving request stream
    (d=16, gamma_k=2^-k, exponential kernel, q=6, rtol=1e-6; eta=2 and the
    Sec. 6.2 weights; N <= args.solve_nmax), all arriving at t=0 and served
    by the continuous-batching server.  lambda=1e-6 needs the float64
    operator (the float32 operator's rounding exceeds lambda by orders of
    magnitude and refinement diverges); float32 + float64-residual
    refinement is compared with float64 at lambda=1e-2.  A Poisson
    offered-load sweep (0.5, 0.8, 1.0 of the closed-loop rate) runs the mixed
    server on a larger sample."""
    reqs = _sample_requests(args.solve_requests, args.solve_nmax)
    sweep = _sample_requests(args.sweep_requests, args.sweep_nmax)
    return {"workload": "serving stream sample: d=16, gamma_k=2^-k, exp kernel, q=6, eta=2, Sec. 6.2 weights, "
                        "leaf 128, rtol=1e-6, all arriving at t=0, 8 active slots",
            "n_range": [min(r.X.shape[0] for r in reqs), max(r.X.shape[0] for r in reqs)],
            "fp64_lambda_1e-6": _serve(reqs, "fp64", 1e-6),
            "fp64_lambda_1e-2": _serve(reqs, "fp64", 1e-2),
            "mixed_lambda_1e-2": _serve(reqs, "mixed", 1e-2),
            "mixed_lambda_1e-2_batched": _serve(reqs, "mixed", 1e-2, batched=True),
            "mixed_lambda_1e-2_poisson": {"n_range": [min(r.X.shape[0] for r in sweep),
                                                      max(r.X.shape[0] for r in sweep)],
                                          **_serve_poisson(sweep, "mixed", 1e-2)},
            "mixed_lambda_1e-2_poisson_batched": {"n_range": [min(r.X.shape[0] for r in sweep),
                                                              max(r.X.shape[0] for r in sweep)],
                                                  **_serve_poisson(sweep, "mixed", 1e-2, batched=True)}}


def run_eta_sweep(args):
    """The bench workload (d = 10 Gaussian, N = 2^20, 16 RHS, mixed) with the
    Sec. 6.2 weight rule and with the bench's rule, each at eta = 0.5 (the
    paper's value) and eta = 1:
    |Lambda|, far blocks, near pairs, matvec time (CUDA events, L2 flushed)
    and the compression error of the mixed matvec against the exact product
    on sampled rows (float64 evaluation of K[rows, :] x)."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    import dwfmm_inputs as di
    from paper_2402_09531_gb300 import Plan
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = workload("mixed")
    if args.n:
        w = di.scaled(w, args.n)
    X, f = di.sites_and_rhs(w)
    Xd = torch.from_numpy(X).to(dev)
    xd = torch.from_numpy(f).to(dev)
    rows = np.sort(np.random.default_rng(11).choice(w.n, size=min(1024, w.n), replace=False))
    # exact K[rows, :] x by float64 evaluation at the sampled sites
    pex = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, q=1.0, eta=1.0, leaf_size=w.leaf,
               precision="fp64", max_rhs=w.nrhs)
    pex.tree_build(Xd)
    exact = torch.zeros((w.nrhs, len(rows)), dtype=torch.float64, device=dev)
    pex.evaluate(torch.from_numpy(np.ascontiguousarray(X[rows])).to(dev), xd, exact)
    torch.cuda.synchronize()
    pex.close()
    exact = exact.cpu().numpy()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": w.name,
           "weights": {"paper_logrho": "Sec. 6.2 rule (tau_k^-1 = eta b_k, b_k = 2 gamma_k)",
                       "inv_gamma": "omega_k = gamma_1 / gamma_k (the bench's rule)"},
           "rows_sampled": int(len(rows)), "etas": {}}
    for rule, eta in (("paper_logrho", 0.5), ("paper_logrho", 1.0), ("inv_gamma", 0.5), ("inv_gamma", 1.0)):
        plan = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, weight_rule=rule, q=w.q,
                    eta=eta, leaf_size=w.leaf, precision="mixed", max_rhs=w.nrhs)
        plan.tree_build(Xd)
        n_x, n_far, n_near, depth = plan.info()
        pairs, diag = near_pairs(plan)
        yd = torch.empty_like(xd)
        for _ in range(2):
            plan.matvec(xd, yd)
        torch.cuda.synchronize()
        times = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.matvec(xd, yd)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        plan.set_profiling(True, serialize=True)
        plan.matvec(xd, yd)
        iso = plan.phase_times(reset=True)
        plan.set_profiling(False)
        y = yd.cpu().numpy()[:, rows]
        col = np.linalg.norm(y - exact, axis=1) / np.linalg.norm(exact, axis=1)
        out["etas"][str(eta) if rule == "paper_logrho" else f"{eta} inv_gamma"] = {
            "weight_rule": rule, "far_engine": plan.far_engine(),
            "n_x": n_x, "far_blocks": n_far, "near_blocks": n_near, "depth": depth,
            "near_pairs": pairs, "near_fraction": pairs / float(w.n) ** 2, "near_engine": plan.near_engine(),
            "matvec_ms": statistics.mean(times), "phase_ms_isolated": {k: v[0] for k, v in iso.items()},
            "throughput_pts_rhs_per_s": w.n * w.nrhs / (statistics.mean(times) / 1e3),
            "compression_error_worst_column": float(col.max()),
            "compression_error_block": float(np.linalg.norm(y - exact) / np.linalg.norm(exact))}
        plan.close()
    print(json.dumps(out), flush=True)


def run_cfg2_solve(args):
    """CG solve of (K_tilde + 1e-6 I) c = f on the float64 d = 8 Matern
    workload (N = 262144, rtol 1e-8): the time per iteration at full size
    (blocking solve capped at a few iterations) and the iteration counts of
    solves of the same shape at smaller N (capped), from which the full solve
    is extrapolated (stated as such).  One JSON line per measurement, as it
    completes."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    import dwfmm_inputs as di
    from paper_2402_09531_gb300 import Plan
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    base = workload("fp64")

    def solve(w, maxit):
        X, f = di.sites_and_rhs(w)
        plan = Plan(d=w.d, kernel=w.kernel, sigma=w.sigma, gamma=w.gamma, q=w.q, eta=w.eta, leaf_size=w.leaf,
                    precision="fp64", max_rhs=1)
        plan.tree_build(torch.from_numpy(X).to(dev))
        fd = torch.from_numpy(f).to(dev)
        cd = torch.zeros_like(fd)
        plan.solve(w.lam, fd, cd, rtol=w.rtol, maxit=2)           # warm-up (workspace)
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, its, rel = plan.solve(w.lam, fd, cd, rtol=w.rtol, maxit=maxit)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        plan.close()
        return {"n": w.n, "status": int(st), "iters": int(its), "relres": float(rel[0]), "s": dt,
                "ms_per_iter": dt * 1e3 / max(1, its)}

    full = solve(base, 20)
    print(json.dumps({"workload": base.name, "lambda": base.lam, "rtol": base.rtol, "full_size": full}), flush=True)
    done = []
    for n in args.cfg2_sizes:
        r = solve(di.scaled(base, n), args.cfg2_maxit)
        print(json.dumps({"size": r}), flush=True)
        if r["status"] == 0:
            done.append((n, r["iters"]))
    if len(done) >= 2:
        ns, its = np.array([a for a, _ in done], dtype=float), np.array([b for _, b in done], dtype=float)
        slope, icpt = np.polyfit(np.log(ns), np.log(its), 1)
        it_full = float(np.exp(icpt) * base.n ** slope)
        print(json.dumps({"extrapolated": {"iterations": it_full, "fit": f"iters ~ N^{slope:.3f}",
                                           "solve_s": it_full * full["ms_per_iter"] / 1e3,
                                           "note": "power law in N through the converged smaller solves, times "
                                                   "the measured full-size time per iteration"}}), flush=True)


def run_batch(args):
    """The batching workload: 256 independent problems (N log-uniform in
    [2048, 65536], d in {6..12}, gamma_k = k^-2, Matern-3/2, q = 5, 1-8
    right-hand sides, float32) as one fused batch matvec (the engine chosen at
    creation: captured launches or one persistent launch; both are timed),
    against the same problems' matvecs one after another.  Throughput
    is sum_p N_p R_p per second; L2 flushed between steps."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import dwfmm_inputs as di
    from paper_2402_09531_gb300 import Batch, Plan
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    probs = di.batching_problems(args.batch_count)
    plans, xs, ys = [], [], []
    t0 = time.perf_counter()
    for w in probs:
        X, f = di.sites_and_rhs(w)
        p = Plan(d=w.d, kernel=w.kernel, gamma=w.gamma, q=w.q, eta=w.eta, leaf_size=w.leaf,
                 precision=args.precision if args.precision != "fp64" else "fp32", max_rhs=w.nrhs)
        p.tree_build(torch.from_numpy(X).to(dev))
        plans.append(p)
        xs.append(torch.from_numpy(f).to(dev))
        ys.append(torch.empty_like(xs[-1]))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = Batch(plans, [w.nrhs for w in probs])
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    units = sum(w.n * w.nrhs for w in probs)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(steps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            z.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(z))
        return statistics.mean(out)

    chosen = b.engine()["engine"]          # the engine creation picked
    try:
        b.set_engine("persistent")           # tuned now if creation did not
    except Exception:
        pass
    eng = b.engine()
    ms_engine = {}
    engines = ["graph", "persistent"] if eng["persistent_available"] else ["graph"]
    for e in engines:
        b.set_engine(e)
        ms_engine[e] = timed(lambda: b.matvec(xs, ys), args.steps)
    b.set_engine(chosen)
    ms_batch = timed(lambda: b.matvec(xs, ys), args.steps)

    def one_by_one():
        for p, x, y in zip(plans, xs, ys):
            p.matvec(x, y)
    ms_seq = timed(one_by_one, max(2, args.steps // 2))
    info = b.info()
    print(json.dumps({
        "workload": f"batching: {len(probs)} problems, N log-uniform in [2048, 65536], d in {{6..12}}, "
                    f"gamma_k = k^-2, Matern-3/2, q = 5, 1-8 RHS, leaf 128",
        "precision": args.precision if args.precision != "fp64" else "fp32",
        "problems": len(probs), "sites": sum(w.n for w in probs), "pts_rhs_per_step": units,
        "batch_ms": ms_batch, "batch_pts_rhs_per_s": units / (ms_batch / 1e3),
        "sequential_ms": ms_seq, "sequential_pts_rhs_per_s": units / (ms_seq / 1e3),
        "speedup": ms_seq / ms_batch, "tree_builds_s": build_s, "batch_create_s": create_s,
        "launch_shape": {
            k: f"{info[k]['threads']} threads per CTA, "
               + ("one launch per right-hand-side class" if info[k]["per_class"] else "one padded launch")
            for k in ("near_shape", "m2l_shape")},
        "autotune_ms": info["tune_ms"], "leaves": info["leaves"],
        "engine": chosen, "engine_ms": ms_engine, "engine_tune_ms": eng["ms"],
        "persistent_launch": eng["persistent_launch"],
        "l2": "flushed between steps (512 MiB write)"}), flush=True)
    b.close()
    for p in plans:
        p.close()


def run_serve_large(args):
    """The serving stream at larger N: the first requests with N in
    [serve_nmin, serve_nmax], float64, lambda = 1e-6, rtol = 1e-6, all
    arriving at t = 0, 8 active slots; p50/p99, solves/s and, per request,
    iterations and time per iteration, from which the largest requests of
    the stream (N = 5e5) are extrapolated (stated as such)."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_09531_gb300.serving import Server, summarize
    torch.cuda.set_device(0)
    reqs = _sample_requests(args.serve_count, args.serve_nmax, args.serve_nmin)
    srv = Server(precision="fp64", max_active=8)
    srv.run(reqs[:1])
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    out = summarize(res, wall)
    srv.close()
    per = []
    byid = {r.rid: r for r in reqs}
    for r in res:
        n = byid[r.rid].X.shape[0]
        busy = (r.t_done - r.t_admit) * 1e3
        per.append({"n": n, "iters": r.iters, "status": r.status, "latency_ms": r.latency_ms,
                    "ms_per_iter_in_mix": busy / max(1, r.iters)})
    out.update({"workload": f"serving stream, N in [{args.serve_nmin}, {args.serve_nmax}], float64, lambda = 1e-6",
                "requests_detail": sorted(per, key=lambda x: x["n"])})
    ok = [p for p in per if p["status"] == "ok"]
    if len(ok) >= 3:
        ns = np.array([p["n"] for p in ok], float)
        it = np.array([p["iters"] for p in ok], float)
        ms = np.array([p["ms_per_iter_in_mix"] for p in ok], float)
        a_it, b_it = np.polyfit(np.log(ns), np.log(it), 1)
        a_ms, b_ms = np.polyfit(np.log(ns), np.log(ms), 1)
        n5 = 5e5
        out["extrapolated_n5e5"] = {"iterations": float(np.exp(b_it) * n5 ** a_it),
                                    "ms_per_iter": float(np.exp(b_ms) * n5 ** a_ms),
                                    "solve_s": float(np.exp(b_it) * n5 ** a_it * np.exp(b_ms) * n5 ** a_ms / 1e3),
                                    "fit": f"iters ~ N^{a_it:.2f}, ms/iter ~ N^{a_ms:.2f} (in an 8-way mix)",
                                    "note": "power laws through the served requests; not measured at N = 5e5"}
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # in a child process with one BLAS thread per core's worker: forking the
    # per-core workers from a process whose BLAS thread pool is running can
    # hang them, and each worker's own threads would oversubscribe the cores
    p = start_oracle_subprocess(args.workload, args.steps, args.warmup)
    res = finish_oracle_subprocess(p, timeout=300.0 + 120.0 * (args.steps + args.warmup))
    if res is None:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle sample did not finish in time"}),
              flush=True)
        return
    w = workload(args.workload)
    value = res["units_per_step"] / res["s_per_step"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["s_per_step"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (uniform sites in prod_k [-gamma_k, gamma_k], N(0,1) right-hand sides)",
        "impl": "reference",
        "config": {"workload": w.name, "d": w.d, "N": w.n, "nrhs": w.nrhs, "kernel": w.kernel, "q": w.q,
                   "leaf": w.leaf, "eta": w.eta},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                         "sample": oracle_sample_text(res, w.nrhs)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="mixed", choices=["mixed", "fp64", "small"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--m2l-engine", default="auto",
                    choices=["auto", "mixed_tf32_tensor", "mixed_symmetric_fp16_tensor"],
                    help="M2L engine of the mixed matvec (auto: timed once per tree)")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--n", type=int, default=0, help="override N (smaller case for profiling)")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the float64 matvec of the same workload (about a minute at N=2^20)")
    ap.add_argument("--solve-requests", type=int, default=8)
    ap.add_argument("--solve-nmax", type=int, default=3000)
    ap.add_argument("--sweep-requests", type=int, default=32)
    ap.add_argument("--sweep-nmax", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-large", action="store_true",
                    help="float64 lambda = 1e-6 serving at larger N, with an extrapolation to N = 5e5")
    ap.add_argument("--serve-nmin", type=int, default=8000)
    ap.add_argument("--serve-nmax", type=int, default=30000)
    ap.add_argument("--serve-count", type=int, default=8)
    ap.add_argument("--batch", action="store_true",
                    help="the 256-problem batching workload: fused batch matvec against one matvec per problem")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--cfg2-solve", action="store_true",
                    help="float64 CG solve of the d = 8 Matern workload: per-iteration time, extrapolation")
    ap.add_argument("--cfg2-sizes", type=int, nargs="*", default=[2048, 4096, 8192, 16384])
    ap.add_argument("--cfg2-maxit", type=int, default=10000)
    ap.add_argument("--eta-sweep", action="store_true",
                    help="the bench workload with the Sec. 6.2 weights at eta = 0.5 and 1 (own JSON line)")
    ap.add_argument("--oracle-sample", default=None)
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample, args.steps, args.warmup)), flush=True)
        return
    if args.eta_sweep:
        run_eta_sweep(args)
    elif args.cfg2_solve:
        run_cfg2_solve(args)
    elif args.batch:
        run_batch(args)
    elif args.serve_large:
        run_serve_large(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
