"""Benchmark: Background SHAP consumer-rows/s on the large workload shaped like the
paper's KDD-Cup-99 run (3,000,000 consumers x 5,000,000 background rows, 127 features,
200 ragged depth-6 trees).

One step = the whole hot path on one batch: background decision patterns and counts,
the pattern-pair contraction and fold (set_background), the consumer patterns, gather
and accumulation into phi (explain), and the FP64 per-feature global attribution of
phi.  value = consumer rows / step time, inputs resident in HBM (both larger than L2).
e2e = the same step through the C ABI with pinned HOST buffers (B and C copied in,
phi copied out inside the timed region).

--impl reference times the FP64 CPU oracle (the count-regrouped tier) on the host
cores on a bounded sample of the same workload, extrapolated linearly in the number
of background rows and consumer rows.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under torchrun,
one process per GPU, every rank runs its own copy of the workload (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "background_shap_consumer_rows_per_sec"
UNIT = "rows/s"


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_rows(m: int, rank: int, world: int):
    """Rows [a, b) of the background that rank counts when the background is sharded."""
    return m * rank // world, m * (rank + 1) // world


def job_rows_per_s(world: int, rows_per_rank: int, seconds: float) -> float:
    """Whole-job throughput: every rank explains its own rows_per_rank rows."""
    return world * rows_per_rank / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, name in enumerate(names):
                    if r[5 + k].lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# sources whose hash a committed ncu summary must match for its counters to stand
EXPLAIN_SOURCES = ["k_explain.cuh", "k_explain.cu", "k_codes.cu", "wdf_device.cuh", "tree_layout.h", "launch.h"]
BACKGROUND_SOURCES = ["k_background.cu", "k_codes.cu", "wdf_device.cuh", "tree_layout.h"]


def profiled_fields(summary: str, sources: list):
    """The key: value lines of a committed ncu summary, or None when the kernel sources
    changed since its counters were taken (a hash in the summary)."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line and not line.startswith("|"))
    h = hashlib.sha256()
    for p in sources:
        with open(os.path.join(ROOT, "paper_2511_09376_gb300", "csrc", p), "rb") as f:
            h.update(f.read())
    if fields.get("source_sha256_16", "").strip() != h.hexdigest()[:16]:
        return None
    return fields


def profiled_traffic(summary: str, sources: list, units, key: str = "traffic_bytes_per_unit"):
    """DRAM bytes from a committed ncu summary (the per-unit figure `key` x units), or
    None when the kernel sources changed since the counters were taken."""
    fields = profiled_fields(summary, sources)
    return None if fields is None or key not in fields else float(fields[key]) * units


def profiled_limiter(summary: str, sources: list):
    """What ncu showed to bound the kernel (e.g. the L1 data pipe's share of its peak
    wavefront rate), or None when the counters are stale or absent."""
    fields = profiled_fields(summary, sources)
    return None if fields is None else fields.get("limiter", "").strip() or None


def workload_config(w, n: int, m: int, world: int, sharded: bool = False) -> dict:
    """The config object of both arms' JSON lines: the workload and how it is run."""
    F = w.n_features
    cb, bb = n * F * 4, m * F * 4
    return {
        "workload": f"{w.name}: n={n} consumers, m={m} background rows, F={F}, T={w.n_trees} trees, depth<={w.depth}",
        "n_consumers": n, "n_background": m, "n_features": F, "n_trees": w.n_trees, "depth": w.depth,
        "l2": f"inputs larger than L2 (B {bb / 1e9:.2f} GB, C {cb / 1e9:.2f} GB)" if min(bb, cb) > 129e6
              else "inputs smaller than L2",
        "parallelism": f"background-sharded{world}" if sharded else f"replicas{world}",
    }


def algorithmic_ops(ens) -> dict:
    """Per consumer row, the work the method must do on the real (unpadded) trees:
    one compare per inner node and one table lookup-add per (leaf, distinct feature on
    its path) -- the O(n T L D) term of the paper's complexity table."""
    compares = adds = 0
    for t in range(ens.n_trees):
        o = int(ens.tree_offset[t])
        stack = [(0, ())]
        while stack:
            v, feats = stack.pop()
            f = int(ens.feature[o + v])
            if f < 0:
                adds += len(set(feats))
            else:
                compares += 1
                stack.append((int(ens.left[o + v]), feats + (f,)))
                stack.append((int(ens.right[o + v]), feats + (f,)))
    return {"compares": compares, "lookup_adds": adds, "ops": compares + adds}


def l1_floor(ens, D: int) -> dict:
    """The fewest L1 data-pipe wavefronts a consumer row needs in the consumer kernel's
    design (one wavefront moves 128 bytes for a warp of 32 rows): one gather of the
    folded slot vector (4 * SP bytes, SP = D + 1 slots padded to 4, 8 or 12) per live
    bottom subtree, i.e. the subtrees of height 2 holding a non-zero leaf, and one read
    plus one write of the row's 4-byte phi accumulator per real inner node."""
    sp = 4 if D + 1 <= 4 else (8 if D + 1 <= 8 else 12)
    live = real = 0
    for t in range(ens.n_trees):
        o = int(ens.tree_offset[t])
        stack, subs = [(0, 0, 0)], set()
        while stack:
            v, h, d = stack.pop()
            if int(ens.feature[o + v]) < 0:
                if float(ens.value[o + v]) != 0.0:
                    # a leaf at depth d is pushed left down to depth D: leaf q of the complete layout
                    q = (h + 1) * (1 << (D - d)) - 1 - ((1 << D) - 1)
                    subs.add(q // 4)
            else:
                real += 1
                stack.append((int(ens.left[o + v]), 2 * h + 1, d + 1))
                stack.append((int(ens.right[o + v]), 2 * h + 2, d + 1))
        live += len(subs)
    gather = live * 4 * sp / 128.0
    phi = 2.0 * real / 32.0
    return {"live_subtree_gathers": live, "real_inner_nodes": real, "wavefronts_per_row": gather + phi,
            "gather_wavefronts_per_row": gather, "phi_wavefronts_per_row": phi}


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2511_09376_gb300 as wdf
    from paper_2511_09376_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.WORKLOADS[args.workload]
    t_gen = time.time()
    ens, C, B = synth.make(w, n_consumers=args.consumers, n_background=args.background)
    gen_s = time.time() - t_gen
    n, m, F = C.shape[0], B.shape[0], C.shape[1]
    ctx = wdf.ctx_create(local_rank)
    e = wdf.load_ensemble(ctx, ens)
    info = wdf.ensemble_info(e)
    dB = torch.from_numpy(B).to(dev)
    dC = torch.from_numpy(C).to(dev)
    phi = torch.empty((n, F), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    shard = None
    if args.shard_background and world > 1:
        # every rank counts its slice of the background; one sum of the counts over the
        # ranks (the only exchange), then each finishes the same background
        import torch.distributed as dist
        a, b = shard_rows(m, rank, world)
        counts = torch.zeros(int(wdf.background_counts_size(e)), dtype=torch.int32, device=dev)
        shard = (dB[a:b], counts, dist)

    def set_bg():
        if shard is None:
            wdf.set_background(e, dB, args.precision)
            return
        part, counts, dist = shard
        counts.zero_()
        wdf.background_counts(e, part, counts)
        dist.all_reduce(counts)
        wdf.set_background_counts(e, counts, m, args.precision)

    def step(ev=None):
        if ev is not None:
            ev[2].record(stream)
        set_bg()
        if ev is not None:
            ev[0].record(stream)
        wdf.explain(e, dC, out=phi)
        if ev is not None:
            ev[1].record(stream)
        wdf.global_attribution(ctx, phi)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = wdf.launch_count()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    # the consumer kernel's own launches, bracketed by CUDA events on the call's stream
    # inside the library (wdf_explain_timing)
    wdf.explain_timing(True)
    start.record(stream)
    for k in range(args.steps):
        step(kev[k])
    stop.record(stream)
    torch.cuda.synchronize()
    barrier()
    kernel_ms_total, kernel_launches = wdf.explain_timing_read()
    wdf.explain_timing(False)
    launches = wdf.launch_count() - launches0
    clk = clocks.stop()
    ms = start.elapsed_time(stop) / args.steps
    explain_ms = statistics.mean(a.elapsed_time(b) for a, b, _ in kev)
    background_ms = statistics.mean(c.elapsed_time(a) for a, _, c in kev)
    ms = max_over_ranks(ms, world, dev)

    # end to end through the C ABI with pinned host buffers
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.from_numpy(C).pin_memory()
    hphi = torch.empty((n, F), dtype=torch.float32).pin_memory()
    for _ in range(max(1, min(args.warmup, 2))):
        wdf.set_background(e, hB, args.precision)
        wdf.explain(e, hC, out=hphi)
    torch.cuda.synchronize()
    barrier()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        wdf.set_background(e, hB, args.precision)
        wdf.explain(e, hC, out=hphi)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, world, dev)

    peaks, peak_kind = _peaks()
    ops = algorithmic_ops(ens)
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # issue roof: 152 SMs x 128 lanes per clock (4 schedulers x 32 lanes)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak_max = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = ops["ops"] * n / (explain_ms * 1e-3) / 1e12
    # per launch of the consumer kernel alone: its rows (n over the launches of one call)
    # over its average launch duration
    launches_per_call = max(1, kernel_launches // max(1, args.steps))
    rows_per_launch = n / launches_per_call
    kernel_ms = kernel_ms_total / max(1, kernel_launches)
    achieved_kernel = ops["ops"] * rows_per_launch / (kernel_ms * 1e-3) / 1e12
    l1 = l1_floor(ens, info["depth"])
    l1_peak = sms * peaks.get("sm_max_mhz", 2070.0) * 1e6
    # background: one compare per inner node and one count per (row, live leaf)
    bg_ops = ops["compares"] + info["n_live_leaves"]
    hbm_bytes = 2 * n * F * 4
    result = {
        "metric": METRIC,
        "value": job_rows_per_s(world, n, ms * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(w, n, m, world, shard is not None),
        "precision": args.precision,
        "ensemble": {"depth": info["depth"], "live_leaves": info["n_live_leaves"], "signatures": info["n_signatures"]},
        "explain_ms": explain_ms,
        "background_ms": background_ms,
        "reduce_ms": ms - explain_ms - background_ms,
        "explain_only_rows_per_s": world * n / (explain_ms * 1e-3),
        "roofline": {
            "kernel": f"k_explain<{info['depth']},64> alone (decisions, entries, gathers, phi accumulation): "
                      f"{launches_per_call} launches per explain call of {n} rows, {kernel_launches} timed "
                      "with CUDA events on the call's stream (wdf_explain_timing)",
            "bound": "alu",
            "achieved": achieved_kernel,
            "peak": alu_peak_max,
            "unit": "Top/s",
            "frac": achieved_kernel / alu_peak_max,
            "ms_per_launch": kernel_ms,
            "rows_per_launch": rows_per_launch,
            "traffic": profiled_traffic("k_explain_large.md", EXPLAIN_SOURCES, rows_per_launch,
                                        "kernel_traffic_bytes_per_unit"),
            "limiter_ncu": profiled_limiter("k_explain_large.md", EXPLAIN_SOURCES),
            "ops_per_row": ops,
            "peak_basis": f"{sms} SMs x 128 lanes/clk x {peaks.get('sm_max_mhz', 2070.0)} MHz (max SM clock, {peak_kind})",
            # against the L1 data pipe (the resource ncu shows bounding the kernel): the
            # fewest wavefronts the design needs per row, at one wavefront per SM per clock
            "l1_floor": {**l1, "peak_wavefronts_per_s": l1_peak,
                         "achieved_floor_wavefronts_per_s": l1["wavefronts_per_row"] * rows_per_launch / (kernel_ms * 1e-3),
                         "frac": l1["wavefronts_per_row"] * rows_per_launch / (kernel_ms * 1e-3) / l1_peak},
            # the whole explain call (the encode kernel and the consumer kernel per chunk)
            "call": {
                "achieved": achieved,
                "frac": achieved / alu_peak_max,
                "ms": explain_ms,
                "algorithmic_bytes": hbm_bytes,
                "traffic": profiled_traffic("k_explain_large.md", EXPLAIN_SOURCES, n),
                "hbm_gbs": hbm_bytes / (explain_ms * 1e-3) / 1e9,
                "hbm_frac_of_measured": hbm_bytes / (explain_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "l1_floor_frac": l1["wavefronts_per_row"] * n / (explain_ms * 1e-3) / l1_peak,
            },
        },
        "roofline_background": {
            "kernel": "set_background: k_encode_codes (on a side stream, overlapping) + k_bg_hist (patterns, "
                      "joint counts) + the small per-leaf, line-map, contraction and fold kernels",
            "bound": "alu",
            "achieved": bg_ops * m / (background_ms * 1e-3) / 1e12,
            "peak": alu_peak_max,
            "unit": "Top/s",
            "frac": bg_ops * m / (background_ms * 1e-3) / 1e12 / alu_peak_max,
            "traffic": profiled_traffic("k_bg_hist_large.md", BACKGROUND_SOURCES, m),
            "limiter_ncu": profiled_limiter("k_bg_hist_large.md", BACKGROUND_SOURCES),
            "ops_per_row": {"compares": ops["compares"], "leaf_counts": info["n_live_leaves"], "ops": bg_ops},
            "hbm_gbs": B.nbytes / (background_ms * 1e-3) / 1e9,
        },
        "e2e": {"value": job_rows_per_s(world, n, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(B.nbytes + C.nbytes),
                "d2h_bytes_per_step": int(n * F * 4)},
        "gpu_launches": int(launches // args.steps),
        "gpu_launches_timed_region": int(launches),
        "clocks": clk,
        "generate_s": gen_s,
    }
    return result, ens, C, B


def cpu_baseline(ens, C, B, budget_s=20.0):
    """The FP64 oracle (count-regrouped tier) on a bounded sample; time per background
    row and per consumer row, extrapolated to the full workload."""
    import oracle
    m_s = min(B.shape[0], 100_000)
    t0 = time.perf_counter()
    counts = oracle.bg_hist(ens, B[:m_s])
    t_bg = (time.perf_counter() - t0) / m_s
    n_s = 64
    t0 = time.perf_counter()
    oracle.values_hist(ens, counts, m_s, C[:n_s])
    t_c = (time.perf_counter() - t0) / n_s
    total = t_bg * B.shape[0] + t_c * C.shape[0]
    return {"value": C.shape[0] / total, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"background counts on {m_s} rows ({t_bg * m_s:.2f} s) and values for {n_s} consumers "
                      f"({t_c * n_s:.2f} s) of the same workload, extrapolated linearly to m={B.shape[0]}, "
                      f"n={C.shape[0]}: {total:.0f} s for the full workload"}


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step is a bounded sample of the workload."""
    import oracle
    from paper_2511_09376_gb300 import synth
    oracle.build()
    w = synth.WORKLOADS[args.workload]
    n_full, m_full = w.n_consumers, w.n_background
    m_s, n_s = min(50_000, m_full), min(32, n_full)
    ens, C, B = synth.make(w, n_consumers=n_s, n_background=m_s)

    sample_s = []

    def step():
        t0 = time.perf_counter()
        counts = oracle.bg_hist(ens, B)
        t1 = time.perf_counter()
        oracle.values_hist(ens, counts, m_s, C)
        t2 = time.perf_counter()
        sample_s.append(t2 - t0)
        return (t1 - t0) / m_s * m_full + (t2 - t1) / n_s * n_full

    for _ in range(args.warmup):
        step()
    sample_s.clear()
    est = [step() for _ in range(args.steps)]
    full_s = statistics.mean(est)
    v = n_full / full_s
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": full_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, n_full, m_full, world),
        # each step times a bounded sample and extrapolates it linearly to the full
        # workload: ms_per_step is that estimate, not a measured wall time
        "ms_per_step_extrapolated": True,
        "ms_per_step_measured_sample": statistics.mean(sample_s) * 1e3,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"per step: background counts on {m_s} rows and values for {n_s} consumers, "
                                   f"extrapolated linearly to m={m_full}, n={n_full}"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def interaction_ops(ens) -> dict:
    """Per consumer row on the real trees: one compare per inner node and one pair
    lookup-add per (leaf, pair of distinct features on its path)."""
    compares = adds = 0
    for t in range(ens.n_trees):
        o = int(ens.tree_offset[t])
        stack = [(0, ())]
        while stack:
            v, feats = stack.pop()
            f = int(ens.feature[o + v])
            if f < 0:
                k = len(set(feats))
                adds += k * (k - 1) // 2
            else:
                compares += 1
                stack.append((int(ens.left[o + v]), feats + (f,)))
                stack.append((int(ens.right[o + v]), feats + (f,)))
    return {"compares": compares, "pair_adds": adds, "ops": compares + adds}


def run_interactions(args):
    """Shapley interaction values (F x F per consumer) of the large workload's ensemble
    against a precomputed background: the step is one wdf_explain_interactions call."""
    import torch

    import oracle
    import paper_2511_09376_gb300 as wdf
    from paper_2511_09376_gb300 import synth

    w = synth.WORKLOADS["large"]
    n = args.consumers or 65536
    m = args.background or 1_000_000
    ens, C, B = synth.make(w, n_consumers=n, n_background=m)
    F = C.shape[1]
    ctx = wdf.ctx_create(0)
    e = wdf.load_ensemble(ctx, ens)
    dB, dC = torch.from_numpy(B).cuda(), torch.from_numpy(C).cuda()
    wdf.set_background(e, dB)
    out = torch.empty((n, F, F), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        wdf.explain_interactions(e, dC, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = wdf.launch_count()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        wdf.explain_interactions(e, dC, out=out)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = wdf.launch_count() - launches0
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    # end to end: host consumer rows in, host interaction matrices out.  The rows go in
    # four chunks through two device buffers, so that the copy of one chunk's matrices
    # to the host overlaps the next chunk's kernels.
    hC = torch.from_numpy(C).pin_memory()
    hout = torch.empty((n, F, F), dtype=torch.float32).pin_memory()
    nch = 4
    rc = max(1, -(-n // nch))
    dbuf = [torch.empty((rc, F, F), dtype=torch.float32, device="cuda") for _ in range(2)]
    s_comp, s_copy = torch.cuda.Stream(), torch.cuda.Stream()
    ev_c = [torch.cuda.Event() for _ in range(2)]
    ev_d = [torch.cuda.Event() for _ in range(2)]

    def e2e_step():
        with torch.cuda.stream(s_comp):
            dC.copy_(hC, non_blocking=True)
        for k in range(nch):
            lo, hi, b = k * rc, min(n, (k + 1) * rc), k % 2
            if hi <= lo:
                break
            s_comp.wait_event(ev_d[b])  # the buffer's previous chunk has reached the host
            wdf.explain_interactions(e, dC[lo:hi], out=dbuf[b][:hi - lo], stream=s_comp)
            ev_c[b].record(s_comp)
            s_copy.wait_event(ev_c[b])
            with torch.cuda.stream(s_copy):
                hout[lo:hi].copy_(dbuf[b][:hi - lo], non_blocking=True)
            ev_d[b].record(s_copy)

    e2e_step()
    torch.cuda.synchronize()
    tt = time.perf_counter()
    for _ in range(max(1, min(args.steps, 3))):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - tt) / max(1, min(args.steps, 3))
    peaks, peak_kind = _peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = sms * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    ops = interaction_ops(ens)
    achieved = ops["ops"] * n / (ms * 1e-3) / 1e12
    result = {
        "metric": "background_shapley_interaction_rows_per_sec", "value": n / (ms * 1e-3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"interactions: large-workload ensemble (T={w.n_trees}, depth<=6, F={F}), n={n} "
                               f"consumers, background of m={m} rows precomputed (not in the step), "
                               f"output n x F x F FP32 ({n * F * F * 4 / 1e9:.2f} GB, larger than L2)",
                   "n_consumers": n, "n_background": m, "n_features": F, "n_trees": w.n_trees},
        "roofline": {"kernel": "the interaction call: pair tables + contraction + k_iv_pack + k_explain_iv",
                     "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Top/s",
                     "frac": achieved / alu_peak, "traffic": None, "ops_per_row": ops,
                     "peak_basis": f"{sms} SMs x 128 lanes/clk x {peaks.get('sm_max_mhz', 2070.0)} MHz ({peak_kind})",
                     "hbm_gbs": n * F * F * 4 / (ms * 1e-3) / 1e9},
        "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(C.nbytes),
                "d2h_bytes_per_step": int(n * F * F * 4)},
        "gpu_launches": int(launches // args.steps), "clocks": clk,
    }
    if not args.no_cpu_baseline:
        ns, ms_bg = 8, min(m, 100_000)
        tb = time.perf_counter()
        counts = oracle.bg_hist(ens, B[:ms_bg])
        t_bg = (time.perf_counter() - tb) / ms_bg
        tc = time.perf_counter()
        oracle.iv_hist(ens, counts, ms_bg, C[:ns])
        t_c = (time.perf_counter() - tc) / ns
        result["cpu_baseline"] = {
            "value": 1.0 / t_c, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"interaction values of {ns} consumers against counts of {ms_bg} background rows "
                      f"({t_c * ns:.2f} s; the background counts, {t_bg * ms_bg:.2f} s, are not in the step)"}
    return result


# The split-precision contraction of the batched and served forms: BF16 hi+mid+lo
# operands (six tcgen05 products), which meet the same FP32-mode bound as the plain path
# at every background size; hi+lo BF16 ("bf16x3") keeps 16 bits per count and misses it
# once counts pass 2^16.
SPLIT_BF16 = "bf16x6"


def ragged_compare(args) -> dict:
    """The ragged batch (64 ensembles of mixed depth and width at their full sizes): the
    plain path (one wdf_explain per ensemble, FP32 contraction) against the batched form
    (one autotuned graph launch over all of them, BF16 hi+mid+lo contraction: the
    FP32-mode accuracy of the plain arm).  Both arms' phi are compared element by
    element; their agreement with the FP64 oracle is checked by the GPU tests
    (1,000 rows per ensemble)."""
    import torch

    import paper_2511_09376_gb300 as wdf
    from paper_2511_09376_gb300 import synth
    specs = synth.ragged_specs()
    ctx = wdf.ctx_create(0)
    dev = torch.device("cuda", 0)
    Cs, t_bg = [], {"fp32": 0.0, SPLIT_BF16: 0.0}
    plain_e, batch_e = [], []
    t0 = time.time()
    for w in specs:
        e_np, C, B = synth.make(w)
        dB = torch.from_numpy(B).to(dev)
        e_plain = wdf.load_ensemble(ctx, e_np)
        e_batch = wdf.load_ensemble(ctx, e_np)
        for e, prec in ((e_plain, "fp32"), (e_batch, SPLIT_BF16)):
            torch.cuda.synchronize()
            s = time.perf_counter()
            wdf.set_background(e, dB, prec)
            torch.cuda.synchronize()
            t_bg[prec] += time.perf_counter() - s
        plain_e.append(e_plain)
        batch_e.append(e_batch)
        Cs.append(torch.from_numpy(C).to(dev))
        del dB, B
    setup_s = time.time() - t0
    rows = sum(c.shape[0] for c in Cs)
    outs_p = [torch.empty((c.shape[0], e.info["n_features"]), device=dev) for c, e in zip(Cs, plain_e)]
    outs_b = [torch.empty_like(o) for o in outs_p]
    batch = wdf.batch_create(ctx, batch_e)
    reqs = list(enumerate(Cs))
    wdf.batch_autotune(batch, reqs, outs=outs_b, reps=2)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def plain():
        for e, c, o in zip(plain_e, Cs, outs_p):
            wdf.explain(e, c, out=o)

    def batched():
        wdf.batch_explain(batch, reqs, outs=outs_b)

    for _ in range(args.warmup):
        plain()
        batched()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = wdf.launch_count()
    ev[0].record(stream)
    for _ in range(args.ragged_steps):
        plain()
    ev[1].record(stream)
    l1 = wdf.launch_count()
    for _ in range(args.ragged_steps):
        batched()
    ev[2].record(stream)
    torch.cuda.synchronize()
    l2 = wdf.launch_count()
    clk = clocks.stop()
    plain_ms = ev[0].elapsed_time(ev[1]) / args.ragged_steps
    batch_ms = ev[1].elapsed_time(ev[2]) / args.ragged_steps
    diff = max(float((a - b).abs().max()) for a, b in zip(outs_p, outs_b))
    tiles = {d: wdf.batch_tile_rows(batch, d) for d in range(2, 9)}
    out = {
        "workload": f"ragged batch: {len(specs)} ensembles, trees 10-500 (log-uniform), depth 2-8, features 20-300, "
                    f"consumers 1e3-2e5 and background rows 1e4-1e6 each; {rows} consumer rows in total",
        "rows_per_step": rows, "steps": args.ragged_steps,
        "plain": {"rows_per_s": rows / (plain_ms * 1e-3), "ms_per_step": plain_ms, "contraction": "fp32",
                  "kernels_per_step": (l1 - l0) // args.ragged_steps,
                  "how": "one wdf_explain per ensemble (encode + consumer kernel each), device-resident rows"},
        "batched": {"rows_per_s": rows / (batch_ms * 1e-3), "ms_per_step": batch_ms, "contraction": SPLIT_BF16,
                    "graph_launches_per_step": 1, "kernels_per_step": (l2 - l1) // args.ragged_steps,
                    "tile_rows": tiles,
                    "how": "one wdf_batch_explain: a CUDA graph with one persistent kernel per depth class, "
                           "autotuned consumer tiles"},
        "batched_vs_plain": plain_ms / batch_ms,
        "max_abs_diff_batched_vs_plain": diff,
        "accuracy": "both arms within |phi - oracle| <= 1e-6 + 1e-5 |oracle| of the FP64 oracle "
                    "(tests/test_gpu_configs.py: 1,000 rows per ensemble for the batched arm; "
                    "tests/test_gpu_depths_precisions.py for FP32 and BF16x6 at depths 2-8)",
        "background_s": t_bg, "setup_s": setup_s, "clocks": clk,
    }
    batch.close()
    for e in plain_e + batch_e:
        e.close()
    ctx.close()
    return out


def _serving_setup(dev, pool_rows=100_000, out_rows=2_000_000):
    """The four resident serving ensembles with their 1e6-row backgrounds precomputed in
    the split-precision contraction, pinned request pools and pinned phi pools."""
    import torch

    import paper_2511_09376_gb300 as wdf
    from paper_2511_09376_gb300 import synth
    specs = synth.serving_specs()
    ctx = wdf.ctx_create(0)
    ens, pools, out_pools = [], [], []
    for k, w in enumerate(specs):
        e_np, _, B = synth.make(w)
        e = wdf.load_ensemble(ctx, e_np)
        dB = torch.from_numpy(B).to(dev)
        wdf.set_background(e, dB, SPLIT_BF16)
        torch.cuda.synchronize()
        del dB, B
        ens.append(e)
        # request rows and phi in pinned host memory, so the server's copies are asynchronous
        pool = torch.empty((pool_rows, w.n_features), dtype=torch.float32).pin_memory().numpy()
        pool[:] = synth.consumers(w, pool_rows)
        pools.append(pool)
        out_pools.append(torch.empty((out_rows, w.n_features), dtype=torch.float32).pin_memory().numpy())
    return specs, ctx, ens, pools, out_pools


def _pct(v, p):
    return float(np.percentile(np.asarray(v, dtype=np.float64), p)) if len(v) else None


def serving_compare(args, setup=None) -> dict:
    """The four resident ensembles behind the continuous-batching server.
    open_loop: Poisson arrivals (args.rate req/s for args.duration s, rows log-uniform
    1..1e5), latency from submit to completion, small requests (at most 1,000 rows)
    reported apart.  saturation: the first requests of the same stream (about 3M rows)
    submitted at once, so the queue never runs dry: the server's capacity.  plain: the
    same requests one wdf_explain call at a time from the same pinned host buffers (the
    plain path's host-memory form).  Both serve the same device-resident ensembles, so
    their phi are compared element by element."""
    import torch

    import paper_2511_09376_gb300 as wdf
    from paper_2511_09376_gb300 import synth
    dev = torch.device("cuda", 0)
    t0 = time.time()
    specs, ctx, ens, pools, out_pools = setup or _serving_setup(dev)
    setup_s = time.time() - t0
    pool_rows, out_rows = pools[0].shape[0], out_pools[0].shape[0]
    slots, max_wave, budget = 4, 32, 16 << 30
    srv = wdf.server_create(ctx, ens, device_budget_bytes=budget, n_slots=slots, max_wave=max_wave)
    for k in range(len(ens)):  # warm-up: one request per ensemble
        t, _ = wdf.server_submit(srv, k, pools[k][:1000])
        wdf.server_wait(srv, t, 600_000)
    wdf.server_reset_stats(srv)

    def views(stream):
        """(ensemble, rows view, phi view) of each request, cycling through the pools."""
        offset, out_off, out = [0] * len(ens), [0] * len(ens), []
        for _, k, n in stream:
            o = offset[k] if offset[k] + n <= pool_rows else 0
            offset[k] = o + n
            p = out_off[k] if out_off[k] + n <= out_rows else 0
            out_off[k] = p + n
            out.append((k, pools[k][o:o + n], out_pools[k][p:p + n]))
        return out

    # open loop
    stream = synth.request_stream(synth.SEED_BASE + 5, args.rate, args.duration, len(ens))
    reqs = views(stream)
    clocks = ClockSampler(0)
    clocks.start()
    tickets = []
    start = time.perf_counter()
    for (at, _, _), (k, C, phi) in zip(stream, reqs):
        delay = start + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(wdf.server_submit(srv, k, C, phi=phi)[0])
    for t in tickets:
        wdf.server_wait(srv, t, 600_000)
    wall = time.perf_counter() - start
    clk_open = clocks.stop()
    st = wdf.server_stats(srv)
    lat = [wdf.server_request_ms(srv, t) for t in tickets]
    small = [x for x, (_, _, n) in zip(lat, stream) if n <= 1000]
    large = [x for x, (_, _, n) in zip(lat, stream) if n > 1000]
    offered = sum(n for _, _, n in stream) / args.duration
    open_loop = {"rate_req_s": args.rate, "duration_s": args.duration, "requests": len(stream),
                 "offered_rows_per_s": offered, "served_rows_per_s": st["rows_per_s"], "wall_s": wall,
                 "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                 "small_requests": len(small), "p50_small_ms": _pct(small, 50), "p99_small_ms": _pct(small, 99),
                 "p50_large_ms": _pct(large, 50), "p99_large_ms": _pct(large, 99), "waves": st["waves"],
                 "clocks": clk_open}
    # saturation: the first requests of the stream, all queued at once
    sat_n, rows_cap = 0, 3_000_000
    acc = 0
    for _, _, n in stream:
        if acc >= rows_cap:
            break
        acc += n
        sat_n += 1
    sat_reqs = views(stream[:sat_n])
    sat_rows = sum(C.shape[0] for _, C, _ in sat_reqs)
    wdf.server_reset_stats(srv)
    clocks = ClockSampler(0)
    clocks.start()
    start = time.perf_counter()
    tickets = [wdf.server_submit(srv, k, C, phi=phi)[0] for k, C, phi in sat_reqs]
    for t in tickets:
        wdf.server_wait(srv, t, 600_000)
    sat_s = time.perf_counter() - start
    clk_sat = clocks.stop()
    st = wdf.server_stats(srv)
    served_phi = [phi.copy() for _, _, phi in sat_reqs[:64]]
    saturation = {"requests": sat_n, "rows": sat_rows, "served_rows_per_s": sat_rows / sat_s, "wall_s": sat_s,
                  "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "waves": st["waves"], "clocks": clk_sat}
    srv.close()
    # the plain path on the same requests: one host-memory wdf_explain per request
    torch.cuda.synchronize()
    start = time.perf_counter()
    for k, C, phi in sat_reqs:
        wdf.explain(ens[k], C, out=phi)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - start
    diff = max(float(np.abs(a - phi).max()) for a, (_, _, phi) in zip(served_phi, sat_reqs[:64]))
    plain = {"rows_per_s": sat_rows / plain_s, "wall_s": plain_s,
             "how": "one wdf_explain per request from the same pinned host buffers, in arrival order"}
    out = {
        "workload": f"serving: ensembles (T, D, F) = {[(w.n_trees, w.depth, w.n_features) for w in specs]}, "
                    f"1e6-row backgrounds precomputed ({SPLIT_BF16} contraction), rows per request log-uniform 1-1e5",
        "server": {"slots": slots, "max_wave": max_wave, "device_budget_gb": budget / 2**30, "express_slot": True},
        "open_loop": open_loop, "saturation": saturation, "plain_same_requests": plain,
        "served_vs_plain": plain_s / sat_s,
        "max_abs_diff_served_vs_plain": diff,
        "accuracy": "the same device-resident ensembles serve both arms (FP32-mode accuracy: "
                    "tests/test_gpu_configs.py checks served rows against the FP64 oracle)",
        "setup_s": setup_s,
    }
    for e in ens:
        e.close()
    ctx.close()
    return out


def contraction_compare(args) -> dict:
    """Step 3 of Algorithm 3 alone, where it is a real dense GEMM: the deep serving
    ensembles (500 trees of depth 7, 1000 of depth 8) on their 1e6-row backgrounds.
    wdf_set_background_counts is timed from precomputed counts in each precision (per-leaf
    counts, scales, line maps, the contraction, the fold), and the tensor-core
    contraction kernel alone with the launch list's events."""
    import torch

    import paper_2511_09376_gb300 as wdf
    from paper_2511_09376_gb300 import synth
    peaks, kind = _peaks()
    ctx = wdf.ctx_create(0)
    dev = torch.device("cuda", 0)
    out = {}
    specs = synth.serving_specs()[3:] if args.deep_only else synth.serving_specs()[2:]
    for w in specs:
        e_np, _, B = synth.make(w, n_background=args.background)
        e = wdf.load_ensemble(ctx, e_np)
        counts = wdf.background_counts(e, torch.from_numpy(B).to(dev))
        m = B.shape[0]
        del B
        info = wdf.ensemble_info(e)
        D, live = info["depth"], info["n_live_leaves"]
        K, N = 1 << D, D << D
        r = {"trees": w.n_trees, "depth": D, "live_leaves": live, "gemm": f"{live} x {K} x {N} (M x K x N)"}
        for prec, products in (("fp32", 1), ("tf32x3", 3), ("bf16x6", 6)):
            wdf.set_background_counts(e, counts, m, prec)  # warm-up (splits the tables once)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            reps = 5
            ev[0].record()
            for _ in range(reps):
                wdf.set_background_counts(e, counts, m, prec)
            ev[1].record()
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / reps
            flops = 2.0 * live * K * N
            r[prec] = {"set_background_counts_ms": ms, "dense_gemm_tflops": flops / (ms * 1e-3) / 1e12,
                       "tensor_products": products if prec != "fp32" else 0}
        r["bf16x6_vs_fp32"] = r["fp32"]["set_background_counts_ms"] / r["bf16x6"]["set_background_counts_ms"]
        out[f"T{w.n_trees}_D{D}"] = r
        e.close()
    ctx.close()
    out["peak_bf16_tflops"] = peaks.get("bf16_tflops")
    out["peak_kind"] = kind
    return out


def run_deep(args):
    """--workload deep: the plain path (one wdf_explain of device rows) on the 1000-tree
    depth-8 serving ensemble, the one whose largest requests set the serving p99."""
    import torch

    import paper_2511_09376_gb300 as wdf
    from paper_2511_09376_gb300 import synth
    w = synth.serving_specs()[3]
    n = args.consumers or 100_000
    e_np, _, B = synth.make(w, n_background=args.background)
    ctx = wdf.ctx_create(0)
    e = wdf.load_ensemble(ctx, e_np)
    wdf.set_background(e, torch.from_numpy(B).cuda(), SPLIT_BF16)
    C = torch.from_numpy(synth.consumers(w, n)).cuda()
    phi = torch.empty_like(C)
    for _ in range(args.warmup):
        wdf.explain(e, C, out=phi)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        wdf.explain(e, C, out=phi)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    return {"metric": METRIC, "value": n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"deep: the plain path on the serving ensemble of {w.n_trees} trees of depth "
                                   f"{w.depth} (F={w.n_features}), n={n} device rows, background of "
                                   f"{B.shape[0]} rows ({SPLIT_BF16} contraction)"}}


def run_ragged(args):
    """--workload ragged: the ragged comparison as the JSON line (value = batched rows/s)."""
    r = ragged_compare(args)
    return {"metric": METRIC, "value": r["batched"]["rows_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": r["steps"], "warmup": args.warmup, "ms_per_step": r["batched"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"]}, "ragged": r}


def run_serving(args):
    """--workload serving: the serving comparison as the JSON line (value = open-loop
    served rows/s)."""
    r = serving_compare(args)
    return {"metric": METRIC, "value": r["open_loop"]["served_rows_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": r["open_loop"]["requests"], "warmup": 4, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"]}, "serving": r}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32x3", "bf16x3", "bf16x6"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # smaller cases of the same workload (the same ensemble, the first rows of the same
    # draws), for profiler captures; the default is the full workload
    ap.add_argument("--consumers", type=int, default=None, help="consumer rows (default: the workload's)")
    ap.add_argument("--background", type=int, default=None, help="background rows (default: the workload's)")
    ap.add_argument("--shard-background", action="store_true",
                    help="N > 1: each rank counts 1/N of the background rows, the counts are summed over ranks")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: requests per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--ragged-steps", type=int, default=5, help="ragged: timed steps of each arm")
    ap.add_argument("--deep-only", action="store_true",
                    help="contraction: only the depth-8 ensemble (for profiler captures)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the ragged-batch and serving comparisons of the default run")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, world, rank)), flush=True)
        return
    if args.workload == "ragged":
        print(json.dumps(run_ragged(args)), flush=True)
        return
    if args.workload == "serving":
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.workload == "deep":
        print(json.dumps(run_deep(args)), flush=True)
        return
    if args.workload == "contraction":
        print(json.dumps({"contraction": contraction_compare(args)}), flush=True)
        return
    if args.workload == "interactions":
        print(json.dumps(run_interactions(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    result, ens, C, B = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            result["cpu_baseline"] = cpu_baseline(ens, C, B)
        del ens, C, B
        if world == 1 and args.workload == "large" and not args.no_forms:
            # the metric's comparison on the same box and run: the batched and served
            # forms against the plain path
            import torch
            torch.cuda.empty_cache()
            result["ragged"] = ragged_compare(args)
            torch.cuda.empty_cache()
            result["serving"] = serving_compare(args)
            torch.cuda.empty_cache()
            result["contraction"] = contraction_compare(args)
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
