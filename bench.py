#!/usr/bin/env python3
"""Benchmark: Striped UniFrac pair x branch updates per second on GB300.

Workload (default): the 113k-shaped one -- a seeded Yule tree with 500,000
tips (999,999 nodes, lengths Exp(mean 0.1)) and 113,000 samples whose
features have prevalence Beta(0.06, 19.94) and heavy-tailed counts
max(1, round(LogNormal(1, 1.5))) (169 M nonzeros); synthetic, generated by
``synth``.  One step = the whole hot path (count levels, embeddings or
presence planes, dense accumulate or tensor-core gram, sparse-row scatter,
diagonal, finalize) for the workload's two methods, unweighted (tcgen05
split-BF16 gram) and weighted_normalized, over the stripe range
[0, 8,192) of 56,500.  Other workloads: ``--workload yule300k_n25000``
(EMP-shaped, all four methods, full matrix), ``yule50k_n2048`` (all four
methods, full matrix), ``batched64``.  ``value`` is pair x branch updates
per second of the mixed path with inputs resident on the GPU; the FP64 path
is measured beside it (on a stripe slice at the large workloads), and the
mixed result's largest difference from the FP64 result is reported over
every value both computed (parity of both paths with the FP64 oracle is the
tests' job).  The oracle runs here only as the CPU baseline and as the
reference arm.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs the same-sized problem (independent
problems, weak scaling, no collective on the data path); rank 0 prints one
JSON line.  ``--impl reference`` times the FP64 CPU oracle (the only
reference this method has) on the host cores on a bounded pair sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair*branch updates/s"
FOUR = ["unweighted", "weighted_unnormalized", "weighted_normalized", "generalized"]
ALL_METHODS = [("unweighted", 1.0), ("weighted_unnormalized", 1.0), ("weighted_normalized", 1.0),
               ("generalized", 0.5), ("unweighted_unnormalized", 1.0), ("vaw_weighted_unnormalized", 1.0),
               ("vaw_weighted_normalized", 1.0)]
METHODS = [ma for ma in ALL_METHODS if ma[0] in FOUR]
# CUDA-core FP32 lanes per SM and the SFU rate per SM on GB300 (sm_103): the
# peaks of the ALU-bound accumulate kernels at the maximum SM clock (the SM
# count is read from the device)
FP32_LANES_PER_SM = 128
SFU_PER_SM = 16
SMS = 152  # replaced by the device's multiprocessor count in run_ours

# per-workload defaults: methods of a step, stripe range [0, stop) (0: all),
# FP32 distance outputs, FP64 comparison slice [0, k) (0: the whole matrix),
# timed steps when --steps is not given (the large workloads' steps take
# seconds: their timed region stays near a minute)
WORKLOAD_DEFAULTS = {
    "yule500k_n113000": dict(methods=["unweighted", "weighted_normalized"], stripe_stop=8192, out_fp32=True,
                             fp64_stripes=64, steps=10),
    "yule300k_n25000": dict(methods=FOUR, stripe_stop=0, out_fp32=False, fp64_stripes=256),
    "yule50k_n2048": dict(methods=FOUR, stripe_stop=0, out_fp32=False, fp64_stripes=0),
    "yule1k_n64": dict(methods=FOUR, stripe_stop=0, out_fp32=False, fp64_stripes=0),
}


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(kernel_key: str, workload: str):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, or
    None when the kernel source changed since the capture or the capture was
    taken on another workload."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as fh:
            d = json.load(fh)
        ent = d.get(kernel_key)
        if not ent or ent.get("workload") != workload:
            return None
        h = hashlib.sha256()
        for src in ent["sources"]:
            with open(os.path.join(ROOT, src), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != ent.get("sources_sha256_16"):
            return None
        return ent["dram_bytes_per_launch_scaled"]
    except (OSError, KeyError, ValueError):
        return None


def oracle_sample_rate(tree_s, table_s, target_seconds: float, seed: int = 99):
    """Oracle throughput on a bounded random pair sample of the workload,
    running the four methods of a step: (updates/s, cores, pairs, seconds)."""
    import oracle
    from synth import pair_subset
    n = table_s.n_samples
    branches = tree_s.n_nodes - 1
    # calibrate on growing samples until one takes an eighth of the target
    probe, dt = 256, 0.0
    while True:
        i, j = pair_subset(n, probe, seed=seed)
        t0 = time.perf_counter()
        for m, a in METHODS:
            oracle.pairs(tree_s, table_s, m, a, i, j)
        dt = max(time.perf_counter() - t0, 1e-3)
        if dt >= target_seconds / 8 or probe >= 200_000:
            break
        probe *= 4
    pairs = int(max(probe, min(400_000, probe * target_seconds / dt)))
    i, j = pair_subset(n, pairs, seed=seed + 1)
    t0 = time.perf_counter()
    used = 1
    for m, a in METHODS:
        used = oracle.pairs(tree_s, table_s, m, a, i, j)[3]
    dt = time.perf_counter() - t0
    return len(METHODS) * i.size * branches / dt, used, int(i.size), dt


def sub_table(table_s, n_sub):
    """The first n_sub samples of a table (same tree, same count recipe)."""
    from synth import Table as STable
    ip = table_s.indptr[: n_sub + 1]
    return STable(n_sub, table_s.n_features, ip.copy(), table_s.indices[: ip[-1]].copy(),
                  table_s.data[: ip[-1]].copy())


def oracle_striped_rate(tree_s, table_s, max_updates_per_thread: float = 1.5e9):
    """The paper's plain striped CPU loop (the oracle's second formulation:
    FP64, host threads over stripes, every branch in postorder) on the stripe
    slice [0, k), one stripe per host thread, for the methods of a step:
    (updates/s, threads, k, seconds, samples).  When one stripe of every
    method is too much work to time within the bench's few minutes, the loop
    runs on the first samples of the table (as many as fit that bound, at
    least 256), labelled as such."""
    import oracle
    branches = tree_s.n_nodes - 1
    n = table_s.n_samples
    if len(METHODS) * n * branches > max_updates_per_thread:
        n_sub = max(256, int(max_updates_per_thread / (len(METHODS) * branches)))
        if n_sub < n:
            table_s = sub_table(table_s, n_sub)
            n = n_sub
    S = n // 2
    if S == 0:
        return None
    k = min(S, oracle.host_cores())
    t0 = time.perf_counter()
    used = 1
    for m, a in METHODS:
        used = oracle.striped(tree_s, table_s, m, a, 0, k)[3]
    dt = time.perf_counter() - t0
    return len(METHODS) * k * n * branches / dt, used, k, dt, n


def run_reference(args, rank, world):
    if rank != 0:  # rank 0 alone times the oracle; the others exit without work
        return 0
    from synth import workload
    tree_s, table_s = workload(args.workload)
    rates, used, pairs = [], 1, 0
    # each step a bounded sample: the whole run stays near two minutes
    per_step = max(1.0, min(args.ref_seconds, 120.0 / (args.warmup + args.steps)))
    for s in range(args.warmup + args.steps):
        r, used, pairs, _ = oracle_sample_rate(tree_s, table_s, per_step, seed=1000 + s)
        if s >= args.warmup:
            rates.append(r)
    value = statistics.mean(rates)
    n = table_s.n_samples
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * len(METHODS) * pairs * (tree_s.n_nodes - 1) / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, tree_s, table_s, l2="n/a (host)"),
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": used, "kind": "oracle",
                         "sample": f"{pairs} random pairs of {n} samples x {len(METHODS)} methods per step "
                                   f"(FP64 per-pair tree walk)"},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, tree_s, table_s, l2):
    stop = getattr(args, "stripe_stop", 0)
    ranged = 0 < stop < table_s.n_samples // 2
    return {"workload": args.workload + (f"[0,{stop})" if ranged else ""),
            "tips": tree_s.n_tips, "nodes": tree_s.n_nodes,
            "samples": table_s.n_samples, "nnz": table_s.nnz,
            "methods": [m for m, _ in METHODS],
            "alpha": 0.5 if any(m == "generalized" for m, _ in METHODS) else None,
            "stripes": "all" if not 0 < getattr(args, "stripe_stop", 0) < table_s.n_samples // 2
            else f"[0, {args.stripe_stop}) of {table_s.n_samples // 2}",
            "sparse_rows_mode": getattr(args, "sparse", 1),
            "sparse_region_bytes": getattr(args, "region_bytes", 0) or "default",
            "sparse_fuse": "default" if getattr(args, "sparse_fuse", -1) < 0 else args.sparse_fuse, "l2": l2}


def max_err_vs_fp64(mixed_outs, fp64_outs):
    """Largest difference of each method's mixed-precision result from the
    FP64 GPU path, over every value of the matrix: absolute, and scaled by
    max(1, |d|) as the unbounded unnormalized method's tolerance is.  (Parity
    of both paths with the FP64 oracle is checked by the tests.)"""
    res = {}
    for (m, _), d32, d64 in zip(METHODS, mixed_outs, fp64_outs):
        diff = np.abs(d32 - d64)
        res[m] = {"max_abs": float(diff.max()) if diff.size else 0.0,
                  "max_scaled": float((diff / np.maximum(1.0, np.abs(d64))).max()) if diff.size else 0.0,
                  "values": int(diff.size)}
    return res


def downstream_agreement(mixed_outs, fp64_outs, sub=512, perms=999):
    """The paper's FP32-vs-FP64 check (Sec. 4): Mantel r^2 between the two
    matrices of each method on all pairs, its permutation p-value on the
    first `sub` samples (`perms` relabellings), and the Procrustes disparity
    of the first 10 principal coordinates."""
    from paper_2005_05826_gb300 import downstream as ds
    res = {}
    for (m, _), d32, d64 in zip(METHODS, mixed_outs, fp64_outs):
        r, _ = ds.mantel(d32, d64, permutations=0)
        s32, s64 = ds.square(d32), ds.square(d64)
        k = min(sub, s64.shape[0])
        iu, ju = np.triu_indices(k, 1)
        _, p = ds.mantel(s32[:k, :k][iu, ju], s64[:k, :k][iu, ju], permutations=perms, seed=1)
        c64, _ = ds.pcoa(d64, k=10)
        c32, _ = ds.pcoa(d32, k=10)
        res[m] = {"mantel_r2": r * r, "mantel_p": p, "p_samples": k, "permutations": perms,
                  "pcoa10_procrustes": ds.procrustes(c64, c32)}
    return res


# FP64 instructions per update of the FP64 accumulate kernels: the min / abs
# kernel one DADD for u - v and one DADD of |u - v| into the accumulator
# (ncu: 2.02); the generalized kernel (alpha = 1/2) 11.07, as ncu counts them
# (smsp__inst_executed_pipe_fp64 per update; profiles/fp64_kernels_yule50k_n2048.md).
FP64_OPS_PER_UPDATE = {"min": 2.0, "gen": 11.07}
# GB300 FP64 lanes per SM and clock: nominal 1.25 TFLOP/s counting an FMA as two
FP64_LANES_PER_SM = 2.0


def fp64_rooflines(f_reps, pairs, sm_max):
    """Roofline objects of the FP64 accumulate kernels from the per-phase
    device times of the FP64 calls: updates of the dense branches over the
    FP64 pipe's instruction rate divided by the instructions per update."""
    out = {}
    for m, r in f_reps:
        if r.acc_launches == 0 or r.t_accumulate_ms <= 0:
            continue
        kind = "gen" if m == "generalized" else "min"
        ach = pairs * r.dense_rows / (r.t_accumulate_ms / 1e3) / 1e12
        obj = {"kernel": "k_stripe_gen<double,4,8>" if kind == "gen" else "k_stripe_min<double,8,8,abs>",
               "bound": "alu", "achieved": ach, "unit": "Tupdates/s"}
        ops = FP64_OPS_PER_UPDATE[kind]
        if ops:
            peak = FP64_LANES_PER_SM * SMS * sm_max * 1e6 / ops / 1e12
            obj.update({"peak": peak, "frac": ach / peak,
                        "peak_basis": f"FP64 pipe {FP64_LANES_PER_SM:g} lanes/clk/SM x {SMS} SMs x "
                                      f"{sm_max:.0f} MHz / {ops:g} FP64 instructions per update"})
        out[f"roofline_{m}"] = obj
    return out


def run_batched(args, rank, world, local_rank):
    """64 uneven tables over one shared 100,000-tip tree: aggregate throughput
    of one batched call per method, plus per-table latency of single calls."""
    import torch

    import paper_2005_05826_gb300 as uf
    from paper_2005_05826_gb300 import build as ufbuild
    from synth import batched_workload

    ufbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    tree_s, tables_s = batched_workload()
    tree = uf.Tree(tree_s.parent, tree_s.length)
    tables = [uf.Table(t.indptr, t.indices, t.data, tree) for t in tables_s]
    branches = tree_s.n_nodes - 1
    pairs = [t.n_samples * (t.n_samples - 1) // 2 for t in tables_s]
    outs = [torch.empty(p, dtype=torch.float64, device=dev) for p in pairs]
    methods = [("unweighted", 1.0), ("weighted_normalized", 1.0)]
    stream = torch.cuda.current_stream(dev)
    uf.uf_set_option("kernel_timing", 0)
    uf.uf_set_option("sparse", args.sparse)

    def step(reps=None):
        for m, a in methods:
            _, r = uf.uf_compute_batch(tree, tables, m, a, "mixed", outs=outs)
            if reps is not None:
                reps.append((m, r))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    times, reps = [], []
    with sampler:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(reps)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    updates_step = len(methods) * sum(pairs) * branches
    value = updates_step * args.steps / sum(times)
    # the same step without CUDA graphs
    uf.uf_set_option("graph", 0)
    step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step()
    e1.record(stream)
    e1.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    uf.uf_set_option("graph", 1)
    # per-table latency: each table alone, both methods
    lat = []
    for t, o in zip(tables, outs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for m, a in methods:
            uf.uf_compute(tree, t, m, a, "mixed", out=o)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
    lat_ms = np.array(lat) * 1e3
    seq_value = updates_step / float(np.sum(lat))
    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Yule tree + iid 1% CSR counts)",
        "config": {"workload": "batched 64 tables, n ~ U{200..5000}, shared 100,000-tip Yule tree",
                   "tables": len(tables), "samples_total": int(sum(t.n_samples for t in tables_s)),
                   "pairs_total": int(sum(pairs)), "methods": [m for m, _ in methods],
                   "l2": "inputs (embedding blocks of GB) larger than L2"},
        "batched_call": {"graph": True, "kernels_per_call": int(reps[0][1][0].kernels),
                         "ms_per_step_without_graph": t_plain * 1e3},
        "per_table_latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                                 "p99": float(np.percentile(lat_ms, 99)),
                                 "max": float(lat_ms.max()),
                                 "sequential_value": seq_value},
        "gpu_launches": int(sum(r[0].kernels for _, r in reps)),
        "clocks": sampler.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2005_05826_gb300 as uf
    from paper_2005_05826_gb300 import build as ufbuild
    from synth import workload

    global SMS
    ufbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    SMS = torch.cuda.get_device_properties(dev).multi_processor_count
    tree_s, table_s = workload(args.workload)
    n = table_s.n_samples
    branches = tree_s.n_nodes - 1
    S = n // 2
    stop = args.stripe_stop if 0 < args.stripe_stop < S else S
    full = stop == S
    # pairs covered per method: all pairs, or the stripe range [0, stop) (stop < S never holds
    # the duplicated half stripe)
    npairs = n * (n - 1) // 2 if full else stop * n
    rng_args = () if full else (0, stop)
    job = None
    if world > 1:
        # the sharded job (stripes are independent subproblems, Abstract and
        # Table 2): rank r computes its own stripe range of the one matrix --
        # [r K, (r + 1) K) with K the one-GPU range, per-rank work fixed, or the
        # whole matrix split evenly once N K stripes would run past it -- with
        # no collective in the timed step; the end-to-end leg gathers every
        # rank's part to rank 0
        from paper_2005_05826_gb300.shard import job_ranges
        job = job_ranges(S, 0 if full else stop, world)
        start, stop = job[rank]
        full = False
        npairs = (stop - start) * n - (n // 2 if 2 * stop == n and stop > start else 0)
        rng_args = (start, stop)
    peaks, peak_src = load_peaks()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # CPU baseline first (before any fork-sensitive GPU state matters)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        r, used, pairs, dt = oracle_sample_rate(tree_s, table_s, args.cpu_seconds)
        cpu = {"value": r, "unit": "updates/s", "cores": used, "kind": "oracle",
               "sample": f"{pairs} random pairs x {len(METHODS)} methods, {dt:.1f} s (FP64 per-pair tree walk)"}
        sl = oracle_striped_rate(tree_s, table_s)
        if sl is not None:
            r, used, k, dt, n_used = sl
            of = f"of {n_used // 2}" if n_used == n else f"of the first {n_used} samples ({n_used // 2} stripes)"
            cpu["striped_loop"] = {
                "value": r, "unit": "updates/s", "cores": used,
                "sample": f"stripes [0, {k}) {of} x {len(METHODS)} methods, {dt:.1f} s (the plain FP64 "
                          f"striped loop, one stripe per thread; from a slice)"}

    tree = uf.Tree(tree_s.parent, tree_s.length)
    table = uf.Table(table_s.indptr, table_s.indices, table_s.data, tree)
    out_dtype = torch.float32 if args.out_fp32 else torch.float64
    n_out = (rng_args[1] - rng_args[0]) * n if rng_args else npairs
    outs = [torch.empty(n_out, dtype=out_dtype, device=dev) for _ in METHODS]  # condensed or stripe-major
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    uf.uf_set_option("kernel_timing", 1)
    uf.uf_set_option("sparse", args.sparse)
    uf.uf_set_option("sparse_region_bytes", args.region_bytes)
    if args.sparse_fuse >= 0:
        uf.uf_set_option("sparse_fuse", args.sparse_fuse)
    uf.uf_set_option("sparse_overlap", args.overlap)

    def step(precision, reps=None):
        for (m, a), o in zip(METHODS, outs):
            _, rep = uf.uf_compute(tree, table, m, a, precision, *rng_args, out=o, out_fp32=args.out_fp32)
            if reps is not None:
                reps.append((m, rep))

    # ---- mixed path: the headline ----
    # The calls run on a stream of their own with device outputs, so each
    # returns once its work is queued and its host work overlaps the previous
    # call's kernels (the null stream would make every call synchronous).
    # Warm-up and the per-phase steps use the option "kernel_timing" (CUDA
    # events per phase, one synchronisation per call); the timed headline
    # steps run without it, as one CUDA graph launch per call.
    run_stream = torch.cuda.Stream(dev)
    stream = run_stream
    with torch.cuda.stream(run_stream):
        for _ in range(args.warmup):
            step("mixed")
        torch.cuda.synchronize()
        uf.uf_set_option("kernel_timing", 0)
        for _ in range(2):  # the graph path's own warm-up
            step("mixed")
        torch.cuda.synchronize()
        times = []
        sampler = ClockSampler(local_rank)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with sampler:
            for _ in range(args.steps):
                flush.zero_()  # L2 flush between steps, outside the timed events
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step("mixed")
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        uf.uf_set_option("kernel_timing", 1)
        # the same steps with per-phase timing: phases, per-kernel rooflines
        # (one step at the large workloads, where a step takes seconds); the
        # scatter runs after the dense kernels here, so that each kernel's
        # time is its own
        uf.uf_set_option("sparse_overlap", 0)
        t_phase, reps = [], []
        phase_steps = args.steps if len(METHODS) * npairs * branches < 5e13 else 1
        for _ in range(phase_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step("mixed", reps)
            e1.record(stream)
            e1.synchronize()
            t_phase.append(e0.elapsed_time(e1))
        uf.uf_set_option("sparse_overlap", args.overlap)
    t_total = sum(times)
    if dist:
        t = torch.tensor([t_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_total = float(t.item())
    updates_step = len(METHODS) * npairs * branches
    job_updates = updates_step
    if dist:  # the whole job's updates: the sum over the ranks' ranges
        u = torch.tensor([float(updates_step)], dtype=torch.float64, device=dev)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        job_updates = float(u.item())
    value = job_updates * args.steps / t_total
    mixed_err = {}  # filled beside the FP64 path when both whole matrices are on the host
    # whole matrices on the host only where the downstream check wants them
    keep_host = full and npairs <= 50_000_000 and not (args.no_downstream and args.no_err)
    mixed_outs = [o.cpu().numpy().astype(np.float64) for o in outs] if keep_host else []
    launches = int(sum(r.kernels for _, r in reps))

    # per-kernel roofline of the accumulate launches (timed inside the steps)
    acc_ms = {}
    sparse = {}
    scat = {}  # per method: region-scatter ms and pair updates over the phase steps
    phases = {}  # device ms per call and phase (CUDA events on the call's stream)
    for m, r in reps:
        d = acc_ms.setdefault(m, [0.0, 0, 0, 0.0, 0, 0, 0])
        d[0] += r.t_accumulate_ms
        d[1] += r.acc_launches
        d[2] += 1
        d[3] += r.exec_flops
        d[4] = r.path
        d[5] = r.dense_rows
        d[6] = r.stripe_tile
        sp = sparse.setdefault(m, {"rows": r.sparse_rows, "dense_rows": d[5], "pairs_at_most": r.sparse_pairs,
                                   "ms_per_call": 0.0})
        sp["ms_per_call"] += r.t_sparse_ms / phase_steps
        if r.sparse_pair_updates > 0:
            sc = scat.setdefault(m, [0.0, 0.0, 0])
            sc[0] += r.t_sparse_ms
            sc[1] += r.sparse_pair_updates
            sc[2] += 1
        ph = phases.setdefault(m, {"embed": 0.0, "accumulate": 0.0, "diagonal": 0.0, "sparse": 0.0,
                                   "finalize": 0.0})
        for key, val in (("embed", r.t_embed_ms), ("accumulate", r.t_accumulate_ms), ("diagonal", r.t_diag_ms),
                         ("sparse", r.t_sparse_ms), ("finalize", r.t_finalize_ms)):
            ph[key] += val / phase_steps
    kern = {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    for m, (ms, nl, ncalls, xflops, path, drows, tile_s) in acc_ms.items():
        per_launch_s = ms / 1e3 / max(nl, 1)
        # algorithmic cell updates of one launch: a call's launches share the
        # call's pairs x the branches that run through the dense kernels (the
        # duplicate half stripe excluded)
        cells = npairs * drows * ncalls / max(nl, 1)
        if path == 1:
            # tensor cores: executed BF16 flops (three split GEMMs, whole
            # 128 x 256 tiles) against the measured dense BF16 peak
            ach = xflops / max(nl, 1) / per_launch_s / 1e12
            peak = float(peaks.get("bf16_tflops", 1900.0))
            kern[m] = {"kernel": "k_gram<tcgen05 kind::f16, 128x256>", "bound": "tensor",
                       "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                       "ms_per_launch": per_launch_s * 1e3, "launches": nl,
                       "peak_basis": f"measured bf16 dense ({peak_src})",
                       "algorithmic_tflops": 2 * cells / per_launch_s / 1e12,
                       "share_of_step": ms / 1e3 / t_total}
            continue
        if m == "generalized":
            # one SFU reciprocal square root per update
            per_clk = SFU_PER_SM
            basis = (f"SFU: {SFU_PER_SM} reciprocal square roots/clk/SM x {SMS} SMs x "
                     f"{sm_max:.0f} MHz (one per update)")
            name = "k_stripe_gen<float,4,8,rsqrt>"
        elif m.startswith("vaw_"):
            # the variance-adjusted weight: one SFU reciprocal square root per update
            per_clk = SFU_PER_SM
            basis = (f"SFU: {SFU_PER_SM} reciprocal square roots/clk/SM x {SMS} SMs x "
                     f"{sm_max:.0f} MHz (one per update)")
            name = "k_stripe_vaw<float,4,4>"
        else:
            # stripes 1, 3, 5, 7 of 8 in the abs form (an FSUB and an FADD of
            # |d| per update, as f32x2 pairs), the others in the min form (an
            # FMNMX on the ALU pipe and an FADD): 1.5 FP32 operations per update
            # on the FMA pipe, whose 128 lanes per clock per SM bound the kernel
            # at 128 / 1.5 updates/clk/SM (the ALU pipe's bound, 64 / 0.5, is higher)
            per_clk = FP32_LANES_PER_SM / 1.5
            basis = (f"FMA pipe: {FP32_LANES_PER_SM} FP32 lanes/clk/SM / 1.5 operations per update x "
                     f"{SMS} SMs x {sm_max:.0f} MHz")
            name = f"k_stripe_min<float,{tile_s // 16},8>"
        peak = per_clk * SMS * sm_max * 1e6 / 1e12
        ach = cells / per_launch_s / 1e12
        kern[m] = {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Tupdates/s",
                   "frac": ach / peak, "ms_per_launch": per_launch_s * 1e3, "launches": nl,
                   "peak_basis": basis, "share_of_step": ms / 1e3 / t_total}
    # the stripe-region scatter (fused lists), timed alone in the phase steps:
    # its pair updates (one 64-bit atomic per accumulator word, counted on the
    # device) against the measured rate of random 64-bit atomics into L2
    if scat:
        l2_peak = uf.uf_probe_l2_atomics(16 << 20)
        for m, (ms, upd, ncalls) in scat.items():
            words = 2 if m == "generalized" else 1
            ach = upd * words / (ms / 1e3)
            kern[m]["scatter"] = {
                "kernel": "k_sparse_region<%s,fused>" % ("presence" if kern[m]["bound"] == "tensor" else "float"),
                "bound": "l2", "achieved": ach / 1e9, "peak": l2_peak / 1e9, "unit": "Gatomics/s",
                "frac": ach / l2_peak, "ms_per_call": ms / ncalls, "pair_updates_per_call": upd / ncalls,
                "peak_basis": "measured in this run: random 64-bit atomic adds into a 16 MB (L2-resident) "
                              "array, uf_probe_l2_atomics",
                "share_of_step": ms / 1e3 / t_total}
    cands = [(kern[m]["share_of_step"], m, kern[m]) for m in kern]
    cands += [(kern[m]["scatter"]["share_of_step"], m, kern[m]["scatter"]) for m in kern if "scatter" in kern[m]]
    _, dom, dom_k = max(cands, key=lambda c: c[0])
    rl = {k: v for k, v in dom_k.items() if k != "scatter"}
    rl["traffic"] = kernel_traffic(rl["kernel"], args.workload if full else f"{args.workload}[0,{stop})")
    rl["method"] = dom

    # ---- e2e through the C ABI: fresh handles from the host arrays (their
    # copy to the device is inside the step), the four calls queued on the
    # stream with device outputs (each call's host work overlaps the previous
    # call's kernels), then every result read back into pinned host memory ----
    e2e = None
    if not args.no_e2e:  # every rank: the job's end-to-end rate at N GPUs
        uf.uf_set_option("kernel_timing", 0)
        host_res = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs]
        # at the large workloads (steps of seconds, results of GB) the
        # device-output variant alone, one warm-up and two timed steps
        large = len(METHODS) * npairs * branches >= 5e13
        modes = (False,) if large else (False, True)
        # pageable result arrays of the host-output variant, allocated (and first
        # touched) once, as a caller keeps its result buffers
        host_arrays = ([] if large else
                       [np.zeros(o.numel(), dtype=np.float32 if args.out_fp32 else np.float64) for o in outs])
        e2e_stream = torch.cuda.Stream(dev)  # a null stream would make every call synchronous
        copy_stream = torch.cuda.Stream(dev)

        def e2e_step(sync_host):
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            tr = uf.Tree(tree_s.parent, tree_s.length)
            t_tree = time.perf_counter()
            tb = uf.Table(table_s.indptr, table_s.indices, table_s.data, tr)
            t_handles = time.perf_counter()
            hb = db = 0.0
            call_s = []
            with torch.cuda.stream(e2e_stream):
                for (m, a), o, ha, h in zip(METHODS, outs, host_arrays or [None] * len(outs), host_res):
                    if sync_host:  # host output: each call returns with its result on the host
                        r, rep = uf.uf_compute(tr, tb, m, a, "mixed", *rng_args, out=ha, out_fp32=args.out_fp32)
                        db += r.nbytes
                    else:
                        _, rep = uf.uf_compute(tr, tb, m, a, "mixed", *rng_args, out=o, out_fp32=args.out_fp32)
                        call_s.append(rep.seconds)
                        # the result's read-back on a copy stream, beside the next call's kernels
                        done = torch.cuda.Event()
                        done.record(e2e_stream)
                        copy_stream.wait_event(done)
                        with torch.cuda.stream(copy_stream):
                            h.copy_(o, non_blocking=True)
                        db += o.numel() * o.element_size()
                    hb += rep.h2d_bytes
                t_queued = time.perf_counter()
            torch.cuda.synchronize()
            stage = (t_handles - t0, t_queued - t_handles, time.perf_counter() - t_queued, t_tree - t0, call_s)
            if dist:  # every rank's part to rank 0: the sharded job's one collective
                from paper_2005_05826_gb300.shard import gather_parts
                for o in outs:
                    gather_parts(dist, n, job, o)
                torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            tb.close()
            tr.close()
            return dt, hb, db, stage

        res = {}
        stages = []  # per e2e step: handles, queueing the calls, the rest until synchronised
        for mode in modes:
            e_times = []
            for s in range((2 if large else max(1, min(args.steps, 3))) + 1):
                dt, h2d, d2h, stage = e2e_step(mode)
                if s > 0:  # the first is a warm-up
                    e_times.append(dt)
                    if not mode:
                        stages.append(stage)
            t_mode = statistics.mean(e_times)
            if dist:  # the slowest rank's step time; bytes of all ranks
                t = torch.tensor([t_mode], dtype=torch.float64, device=dev)
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                t_mode = float(t.item())
            res[mode] = (t_mode, world * h2d, world * d2h)
        t_e, h2d, d2h = res[False]
        e2e = {"value": job_updates / t_e, "unit": "updates/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * t_e,
               "path": f"fresh tree and table handles from the host arrays, {len(METHODS)} uf_compute calls "
                       f"queued on the stream with device outputs, each result read into pinned host memory "
                       f"on a copy stream beside the next call's kernels",
               "ms_stages": {"handles": 1e3 * statistics.mean(x[0] for x in stages),
                             "tree_handle": 1e3 * statistics.mean(x[3] for x in stages),
                             "queue_calls": 1e3 * statistics.mean(x[1] for x in stages),
                             "calls_host": [1e3 * statistics.mean(x[4][i] for x in stages)
                                            for i in range(len(stages[0][4]))],
                             "device_and_copies": 1e3 * statistics.mean(x[2] for x in stages)}}
        if True in res:
            e2e["host_output_calls"] = {"value": job_updates / res[True][0],
                                        "ms_per_step": 1e3 * res[True][0],
                                        "d2h_bytes_per_step": int(res[True][2]),
                                        "path": "the same with pageable host result arrays the caller reuses "
                                                "(each call returns synchronously)"}
        uf.uf_set_option("kernel_timing", 1)

    # ---- FP64 path beside it ----
    fp64 = None
    if rank == 0 and not args.no_fp64 and args.fp64_stripes > 0:
        # FP64 path on the stripe slice [0, fp64_stripes) only (large workloads)
        S = uf.uf_stripe_count(n)
        k = min(args.fp64_stripes, S - 1)
        sl = torch.empty(k * n, dtype=torch.float64, device=dev)
        # an untimed pass (each method's first FP64 call: its split and
        # tuning) that also compares the mixed result on the same cells
        # (stripe-major range output, or gathered from the condensed full
        # output); then a timed pass
        for m, a in METHODS:
            uf.uf_compute(tree, table, m, a, "fp64", 0, k, out=sl)
            if full:
                cs = torch.arange(k * n, device=dev, dtype=torch.int64)
                ss, kk = cs // n, cs % n
                jj = (kk + ss + 1) % n
                lo, hi = torch.minimum(kk, jj), torch.maximum(kk, jj)
                mixed_sl = outs[METHODS.index((m, a))][n * lo - lo * (lo + 1) // 2 + (hi - lo - 1)]
            else:
                mixed_sl = outs[METHODS.index((m, a))][: k * n]
            diff = (mixed_sl.double() - sl).abs()
            mixed_err[m] = {"max_abs": float(diff.max()),
                            "max_scaled": float((diff / torch.clamp(sl.abs(), min=1.0)).max()),
                            "values": int(diff.numel()), "on": f"stripes [0, {k})"}
        f_reps = []
        torch.cuda.synchronize()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for m, a in METHODS:
            _, rep = uf.uf_compute(tree, table, m, a, "fp64", 0, k, out=sl)
            f_reps.append((m, rep))
        e1.record(stream)
        e1.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        upd = sum(r.updates for _, r in f_reps)
        fp64 = {"value": upd / t64, "unit": "updates/s", "ms_for_slice": t64 * 1e3,
                "slice": f"stripes [0, {k}) of {S}, all methods of the step (from a slice)",
                "ms_per_method": {m: r.t_accumulate_ms + r.t_diag_ms + r.t_embed_ms + r.t_finalize_ms
                                  for m, r in f_reps}}
        fp64.update(fp64_rooflines(f_reps, k * n, sm_max))
        if full and not args.no_downstream:
            # the paper's FP32-vs-FP64 check (Sec. 4) on a sample subset: the
            # mixed full matrix's entries of the first `sub` samples against
            # the FP64 path on those samples (a pair's distance depends on its
            # two samples only)
            sub = min(n, 2000)
            sub_s = sub_table(table_s, sub)
            tsub = uf.Table(sub_s.indptr, sub_s.indices, sub_s.data, tree)
            iu, ju = np.triu_indices(sub, 1)
            idx = torch.as_tensor(n * iu - iu * (iu + 1) // 2 + (ju - iu - 1), device=dev)
            mixed_sub = [o[idx].double().cpu().numpy() for o in outs]
            fp64_sub = [uf.uf_compute(tree, tsub, m, a, "fp64")[0] for m, a in METHODS]
            fp64["downstream_vs_mixed"] = downstream_agreement(mixed_sub, fp64_sub, sub=sub)
            fp64["downstream_on"] = (f"the first {sub} samples: entries of the mixed full matrix against "
                                     f"the FP64 path on those samples")
            tsub.close()
    elif rank == 0 and not args.no_fp64:
        step("fp64")
        torch.cuda.synchronize()
        f_reps = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        step("fp64", f_reps)
        e1.record(stream)
        e1.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        fp64_outs = [o.cpu().numpy().astype(np.float64) for o in outs] if keep_host else []
        per_method = {m: r.t_accumulate_ms + r.t_diag_ms + r.t_embed_ms + r.t_finalize_ms
                      for m, r in f_reps}
        fp64 = {"value": updates_step / t64, "unit": "updates/s", "ms_per_step": t64 * 1e3,
                "ms_per_method": per_method}
        fp64.update(fp64_rooflines(f_reps, npairs, sm_max))
        if keep_host and not args.no_err:
            mixed_err = max_err_vs_fp64(mixed_outs, fp64_outs)
        if keep_host and not args.no_downstream:
            fp64["downstream_vs_mixed"] = downstream_agreement(mixed_outs, fp64_outs)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    clocks = sampler.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Yule tree + Beta-prevalence CSR counts)",
        "config": workload_config(args, tree_s, table_s, l2="flushed between steps (256 MB write)"),
        "precision": "mixed: FP32 updates (unweighted: exact 0/1 x split-BF16 lengths on tcgen05, "
                     "FP32 accumulation), int64 fixed-point accumulators, FP64 division",
        "max_abs_err_vs_fp64": max((v["max_abs"] for v in mixed_err.values()), default=None),
        "max_err_vs_fp64": mixed_err or None,
        "updates_basis": "dense-equivalent: every sample pair x every non-root branch per method, "
                         "including the zero terms that the sparse-row path skips",
        "roofline": rl,
        "kernels": kern,
        "sparse_rows": sparse,
        "phases_ms_per_call": phases,
        "ms_per_step_with_phase_timing": statistics.mean(t_phase) if t_phase else None,
        "timing": "the four calls queued on a non-default stream with device outputs (each returns once "
                  "enqueued; one CUDA graph per call); CUDA events on that stream around each step; the "
                  "per-phase step (phases, kernel rooflines) runs the scatter after the dense kernels",
        "peak_source": peak_src,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "fp64_path": fp64,
        "mixed_vs_fp64_speedup": (value / fp64["value"]) if fp64 else None,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20, or 10 for the 113k-shaped workload)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="yule500k_n113000",
                    help="yule500k_n113000 (default; 113k-shaped), yule300k_n25000 (EMP-shaped), "
                         "yule50k_n2048, yule1k_n64, batched64")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer run")
    ap.add_argument("--fp64-stripes", type=int, default=-1,
                    help="run the FP64 comparison on stripes [0, K) only (0: the whole matrix; "
                         "default: per workload)")
    ap.add_argument("--no-err", action="store_true", help="skip the comparison of the mixed and FP64 results")
    ap.add_argument("--methods", default="default",
                    help="comma list of methods per step (any of the seven), or all (the four base "
                         "methods); default: the workload's methods")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-downstream", action="store_true",
                    help="skip the Mantel / principal-coordinate agreement of the mixed and FP64 matrices")
    ap.add_argument("--out-fp32", type=int, choices=[0, 1], default=-1,
                    help="FP32 distance outputs, halving the output memory of very large runs "
                         "(default: per workload)")
    ap.add_argument("--stripe-stop", type=int, default=-1,
                    help="time the stripe range [0, K) of every method instead of all stripes "
                         "(0: all; default: per workload)")
    ap.add_argument("--region-bytes", type=int, default=0,
                    help="option sparse_region_bytes (0: the library default)")
    ap.add_argument("--sparse-fuse", type=int, choices=[-1, 0, 2, 6], default=-1,
                    help="option sparse_fuse (-1: the library default)")
    ap.add_argument("--overlap", type=int, choices=[0, 1], default=1,
                    help="option sparse_overlap: sparse scatter beside the dense kernel")
    ap.add_argument("--sparse", type=int, choices=[0, 1, 2], default=1,
                    help="sparse-row path: 0 every branch dense, 1 cost model (default), 2 every branch that fits")
    args = ap.parse_args()
    dflt = WORKLOAD_DEFAULTS.get(args.workload, WORKLOAD_DEFAULTS["yule50k_n2048"])
    if args.steps is None:
        args.steps = dflt.get("steps", 20)
    if args.stripe_stop < 0:
        args.stripe_stop = dflt["stripe_stop"]
    if args.fp64_stripes < 0:
        args.fp64_stripes = dflt["fp64_stripes"]
    args.out_fp32 = dflt["out_fp32"] if args.out_fp32 < 0 else bool(args.out_fp32)
    want = (dflt["methods"] if args.methods == "default" else
            FOUR if args.methods == "all" else args.methods.split(","))
    METHODS[:] = [ma for ma in ALL_METHODS if ma[0] in want]
    if not METHODS:
        ap.error(f"no known method in {args.methods!r}")
    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched64":
        return run_batched(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
