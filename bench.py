#!/usr/bin/env python3
"""Benchmark: single-source SimRank queries/s on R-MAT scale 20 at eps = 0.02.

Workload (synthetic, seeded): directed R-MAT graph, scale 20 (n = 1,048,576),
edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), deduplicated, no
self-loops, int32 in-neighbour CSR; c = 0.6, eps = 0.02 (z = ln(2n) /
(2 (eps - 3/n)^2)), 64 uniformly drawn sources, one query per launch.  A step
is one full query (steps a1-a5) for the next source of the list.

A step is one pass over all 64 sources (64 queries), so the timed set does
not depend on the step count.  Timing: W untimed warm-up passes, then K timed
ones.  Every query is timed with CUDA events on its stream; the 256 MB L2
flush written between queries lies outside those intervals.  The dominant
kernel (target walks, step a4) is timed with events the library records
around its launch.  ``e2e`` repeats the K passes through the same C-ABI call
with host output buffers, so the timed region includes the device-to-host
copy of every score vector.  The roofline block names the bound that binds:
with the adjacency inside the L2 it is the random-gather rate measured live
by the probe on an array of the adjacency's size (the HBM-copy fraction is
kept beside it, labelled).

``--impl reference`` times the CPU oracle (the plain C restatement of the
method, OpenMP over targets on the host cores) on a bounded sample of the same
workload and prints the same JSON line with ``"impl": "reference"``.

Multi-GPU (torchrun): every rank runs its own 64-source list with no
data-path collective (weak scaling); rank 0 prints the aggregate.
``--workload split`` instead splits every query over the ranks by target
range (the owner rule of Section 5.5) and all-gathers the score slices.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

C = 0.6
EPS = 0.02
SCALE = 20
N_SOURCES = 64
GRAPH_SEED = 1
SOURCE_SEED = 2
QUERY_SEED = 20240405
BYTES_PER_STEP = 12   # algorithmic: 8 B row_ptr pair of the current node + 4 B in-neighbour entry
METRIC = "single-source SimRank queries/s at eps=0.02; walk steps/s vs gather roofline"
WORKLOAD = "rmat20_ef16_eps0.02_64src_one_query_per_launch"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3,
                    help="timed steps; a step is one pass over the 64 sources")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="approximate CPU time budget of the oracle baseline")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-probe", action="store_true")
    ap.add_argument("--workload", default="plain",
                    choices=["plain", "batch", "linear", "serve", "probe", "split"],
                    help="plain: the R-MAT 20 one-query-per-launch workload; batch: "
                         "batched multi-source on R-MAT --batch-scale vs the plain path")
    ap.add_argument("--batch-scale", type=int, default=24)
    ap.add_argument("--literal-shuffle", action="store_true",
                    help="plain workload with every target's walks shuffled too")
    ap.add_argument("--warmup-rule", action="store_true",
                    help="plain workload with the warm-up algorithm's sample size and truncation")
    ap.add_argument("--layout", default=None, choices=["narrow", "wide", "csr"],
                    help="adjacency entry layout (default: chosen by graph size)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: offered requests/s")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-budget-mb", type=int, default=1024)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-target-ms", type=float, default=1000.0,
                    help="serve: latency target of the admission (0: memory only, FIFO)")
    ap.add_argument("--batch-sources", type=int, default=12,
                    help="sources of the 4096-source batching list that are run")
    ap.add_argument("--batch-eps", type=float, default=0.0,
                    help="batch: one eps for every source instead of the list's mixed eps")
    ap.add_argument("--topk", type=int, default=0,
                    help="batch: return each source's top-k targets (srk_multi_source_topk) "
                         "instead of dense rows; the plain comparison is skipped")
    ap.add_argument("--shared-walks", action="store_true",
                    help="batch: target walks drawn once for all sources of a batch "
                         "(SRK_OPT_SHARED_WALKS), against one query per launch with the "
                         "same flag")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, pg, device) -> float:
    """The slowest rank's time (all_reduce MAX); identity on one rank."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def make_workload():
    from srk_inputs import rmat_in_csr, uniform_sources
    rp, col = rmat_in_csr(SCALE, seed=GRAPH_SEED)
    n = rp.size - 1
    sources = uniform_sources(n, N_SOURCES, seed=SOURCE_SEED)
    return rp, col, sources


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gather_probe(srk, torch, dev, n_words, cache_ops=(0,)):
    """Random 4-byte gather rate (loads/s) on an n_words int32 array, for each
    PTX cache operator in cache_ops (SRK_PROBE_*); returns a list of rates."""
    data = torch.randint(0, 1 << 30, (n_words,), dtype=torch.int32, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    rates = []
    for op in cache_ops:
        srk.srk_probe_gather(data, 64, 1, sink, cache_op=op)
        torch.cuda.synchronize()
        iters, rate = 500, 0.0
        for rep in range(3):
            ev[0].record()
            loads = srk.srk_probe_gather(data, iters, 11 + rep, sink, cache_op=op)
            ev[1].record()
            ev[1].synchronize()
            t = ev[0].elapsed_time(ev[1]) / 1e3
            rate = max(rate, loads / t) if rep else rate
            if rep == 0:
                iters = max(100, int(iters * 0.05 / t))
        rates.append(rate)
    del data
    return rates


def variant_name(args):
    """The estimator variant of the plain workload's queries."""
    if args.literal_shuffle and args.warmup_rule:
        return "literal shuffle + warm-up sample rule"
    if args.literal_shuffle:
        return "literal shuffle (every target's walks shuffled, Section 5.2)"
    if args.warmup_rule:
        return "warm-up sample rule (Section 3)"
    return "paper defaults (source walks shuffled)"


def variant_suffix(args):
    return ("_literal" if args.literal_shuffle else "") + ("_warmup" if args.warmup_rule else "")


def kernel_source_sha256():
    """sha256 over the code the target-walk kernel is compiled from and the
    code that lays out the adjacency it reads (the kernel file, the device
    header, the graph loader), with comments and whitespace removed, so that
    an edit of the prose alone keeps a traffic record valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in ("srk_query.cu", "srk_device.cuh", "srk_graph.cu"):
        with open(os.path.join(ROOT, "paper_2304_04015_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def recorded_profile():
    """The committed ncu record of the target-walk kernel, if it was taken on
    the current kernel sources, else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_target_walks_rmat20_traffic.json")) as f:
            rec = json.load(f)
        return rec if rec.get("kernel_sources_sha256") == kernel_source_sha256() else None
    except Exception:
        return None


def recorded_traffic():
    """DRAM bytes per target-walk step of the target-walk kernel, from the
    committed ncu summary, if it was taken on the current kernel sources."""
    rec = recorded_profile()
    if rec is None:
        return None
    return float(rec["dram_bytes_per_launch"]) / float(rec["target_steps_of_launch"])


def recorded_l2_sectors():
    """L2 sectors requested by L1 per target-walk step (ncu, current sources)."""
    rec = recorded_profile()
    if rec is None or "l2_sectors_from_l1_of_launch" not in rec:
        return None
    return float(rec["l2_sectors_from_l1_of_launch"]) / float(rec["target_steps_of_launch"])


def cpu_baseline(rp, col, sources, budget_s, **variant):
    """The oracle as it stands, on the host cores, on a bounded target sample
    (``variant``: the literal_shuffle / warmup_rule options of the queries)."""
    from oracle import sampler
    n = rp.size - 1
    s = int(sources[0])
    rng = np.random.default_rng(7)
    threads = os.cpu_count() or 1
    k = 2048
    while True:
        targets = np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        res = sampler.run(rp, col, n, s, C, EPS, QUERY_SEED, targets=targets, threads=threads,
                          **variant)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 4 or k >= n:
            break
        k = min(n, int(k * max(2.0, budget_s / max(dt, 1e-3) / 2)))
    per_query = dt * n / k
    steps = int(res.steps.sum()) * n / k
    return {"value": 1.0 / per_query, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": "source %d, %d of %d targets (uniform sample), %.1f s; "
                      "queries/s scaled by n/targets" % (s, k, n, dt),
            "steps_per_s": steps / per_query}


def cpu_baseline_mix(graphs_np, queries, budget_s):
    """The oracle as it stands on a mix of queries [(graph index, s, eps)]:
    each query on a uniform target sample grown until it takes about its
    share of budget_s, its time scaled by n/targets; returns queries/s over
    the mix (total scaled time / number of queries)."""
    from oracle import sampler
    rng = np.random.default_rng(7)
    threads = os.cpu_count() or 1
    share = budget_s / max(1, len(queries))
    total, parts = 0.0, []
    for gi, s, eps in queries:
        rp, col = graphs_np[gi]
        n = rp.size - 1
        k = min(n, 256)
        while True:
            targets = np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)
            t0 = time.perf_counter()
            sampler.run(rp, col, n, int(s), C, float(eps), QUERY_SEED, targets=targets,
                        threads=threads)
            dt = time.perf_counter() - t0
            if dt >= share / 4 or k >= n:
                break
            k = min(n, int(k * max(2.0, share / max(dt, 1e-3) / 2)))
        total += dt * n / k
        parts.append("n=%d s=%d eps=%g: %d targets %.1f s" % (n, s, eps, k, dt))
    return {"value": len(queries) / total, "unit": "queries/s", "cores": threads,
            "kind": "oracle", "sample": "; ".join(parts) + "; times scaled by n/targets"}


def run_batch(args, rank, world):
    """Batched multi-source (srk_multi_source, one persistent launch per
    batch) against the plain path (one srk_single_source per source) on the
    same sources and eps: R-MAT scale --batch-scale, 4096 sources of which a
    third have top in-degree, a third median in-degree and a third none,
    eps per source from {0.05, 0.02, 0.01}; the first --batch-sources of the
    list interleaved by group are run."""
    import torch
    from srk_inputs import rmat_in_csr_torch, mixed_sources, mixed_eps
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as srk
    t0 = time.perf_counter()
    rp_d, col_d = rmat_in_csr_torch(args.batch_scale, seed=GRAPH_SEED, device=dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    rp = rp_d.cpu().numpy()
    n, m = rp.size - 1, int(col_d.numel())
    all_src = mixed_sources(rp, 4096, seed=3)
    all_eps = mixed_eps(4096, seed=3)
    third = 4096 // 3
    order = [g * third + i for i in range(third) for g in range(3)]
    order += list(range(3 * third, 4096))  # the last group's extra source
    pick = order[:args.batch_sources]
    sources = [int(all_src[i]) for i in pick]
    eps = [float(all_eps[i]) for i in pick]
    if args.batch_eps > 0:
        eps = [args.batch_eps] * len(sources)
    g = srk.srk_graph_load(rp_d, col_d, layout=args.layout)
    k = len(sources)
    if args.topk > 0:
        return run_batch_topk(args, srk, torch, dev, g, rp, n, m, sources, eps, pick, t_gen)
    out = torch.empty((k, n), dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sw = args.shared_walks
    # warm-up: the first call autotunes the persistent kernel's launch shape
    srk.srk_multi_source(g, sources[:3], C, eps[:3], QUERY_SEED, out[:3], shared_walks=sw)
    torch.cuda.synchronize()
    st = srk.SrkStats()
    ev[0].record()
    srk.srk_multi_source(g, sources, C, eps, QUERY_SEED, out, stats=st, shared_walks=sw)
    ev[1].record()
    ev[1].synchronize()
    t_batch = ev[0].elapsed_time(ev[1]) / 1e3
    single = torch.empty(n, dtype=torch.float64, device=dev)
    t_plain, same, plain_steps = 0.0, True, 0
    for i, s in enumerate(sources):
        pst = srk.SrkStats()
        srk.srk_single_source(g, s, C, eps[i], QUERY_SEED, single, stats=pst, shared_walks=sw)
        plain_steps += pst.target_steps
        torch.cuda.synchronize()
        ev[0].record()
        srk.srk_single_source(g, s, C, eps[i], QUERY_SEED, single, shared_walks=sw)
        ev[1].record()
        ev[1].synchronize()
        t_plain += ev[0].elapsed_time(ev[1]) / 1e3
        same = same and bool(torch.equal(single, out[i]))
    deg = np.diff(rp)
    peak, peak_kind = load_peaks()
    achieved = st.target_steps * BYTES_PER_STEP / t_batch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": "kb_target_walks",
                "peak_kind": peak_kind + " (HBM copy)", "bytes_per_unit": BYTES_PER_STEP,
                "unit_name": "target-walk step",
                "note": "whole batch time (the source phases are a few percent)"}
    gather = None
    if not args.skip_probe:
        probe = gather_probe(srk, torch, dev, n + m)[0]
        gather = {"probe_gathers_per_s_graph_sized": probe,
                  "kernel_steps_per_s": st.target_steps / t_batch,
                  "frac_of_graph_sized_probe": st.target_steps / t_batch / probe}
    base = None
    if not args.no_cpu_baseline:
        col_h = col_d.cpu().numpy()
        mix = [(0, sources[i], eps[i]) for i in range(min(3, k))]
        base = cpu_baseline_mix([(rp, col_h)], mix, args.cpu_seconds)
        del col_h
    line = {"metric": "batched multi-source queries/s (R-MAT scale %d, mixed eps)" % args.batch_scale,
            "workload": "batch_rmat%d_mixed_sources_%s%s" % (
                args.batch_scale, "eps%g" % args.batch_eps if args.batch_eps > 0 else "mixed_eps",
                "_shared_walks" if sw else ""),
            "shared_walks": sw, "plain_target_steps": plain_steps,
            "value": k / t_batch, "unit": "queries/s", "higher_is_better": True,
            "plain_value": k / t_plain, "batched_over_plain": t_plain / t_batch,
            "identical_to_plain": same, "sources": k, "n": n, "m": m,
            "source_in_degrees": [int(deg[s]) for s in sources], "eps": eps,
            "target_steps": st.target_steps, "walk_steps_per_s": st.target_steps / t_batch,
            "batch_shape": st.batch_shape, "graph_gen_s": t_gen,
            "adjacency": srk.srk_graph_layout(g),
            "roofline": roofline, "gather_roofline": gather, "cpu_baseline": base,
            "note": "subset of the 4096-source list; the full list is ~1e15 walk steps"}
    print(json.dumps(line), flush=True)
    g.close()
    return 0


def run_batch_topk(args, srk, torch, dev, g, rp, n, m, sources, eps, pick, t_gen):
    """The batching list through the sparse output: every source's top-k
    targets (srk_multi_source_topk), timed with CUDA events over the whole
    call; no dense k x n matrix exists at any time."""
    k, top = len(sources), args.topk
    tn = torch.empty((k, top), dtype=torch.int32, device=dev)
    ts = torch.empty((k, top), dtype=torch.float64, device=dev)
    tc = torch.empty(k, dtype=torch.int32, device=dev)
    nz = torch.empty(k, dtype=torch.int64, device=dev)
    sw = args.shared_walks
    srk.srk_multi_source_topk(g, sources[:3], C, eps[:3], QUERY_SEED, top, tn[:3], ts[:3],
                              shared_walks=sw)   # warm-up (autotuner)
    torch.cuda.synchronize()
    st = srk.SrkStats()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    srk.srk_multi_source_topk(g, sources, C, eps, QUERY_SEED, top, tn, ts, tc, nz, stats=st,
                              shared_walks=sw)
    ev[1].record()
    ev[1].synchronize()
    t = ev[0].elapsed_time(ev[1]) / 1e3
    deg = np.diff(rp)
    groups = {"top in-degree": 0, "median in-degree": 0, "no in-neighbours": 0}
    third = 4096 // 3
    for i in pick:
        groups[("top in-degree", "median in-degree", "no in-neighbours")[min(2, i // third)]] += 1
    nzh = nz.cpu().numpy()
    line = {"metric": "batched multi-source queries/s with top-%d output (R-MAT scale %d, "
                      "mixed eps)" % (top, args.batch_scale),
            "workload": "batch_rmat%d_mixed_sources_mixed_eps_top%d%s"
                        % (args.batch_scale, top, "_shared_walks" if sw else ""),
            "value": k / t, "unit": "queries/s", "higher_is_better": True, "seconds": t,
            "sources": k, "source_groups": groups, "eps_counts": {str(e): eps.count(e) for e in
                                                                  sorted(set(eps))},
            "n": n, "m": m, "top": top, "target_steps": st.target_steps,
            "walk_steps_per_s": st.target_steps / t,
            "nnz_per_source": {"min": int(nzh.min()), "median": float(np.median(nzh)),
                               "max": int(nzh.max())},
            "output_bytes": k * top * 12, "dense_bytes_avoided": k * n * 8,
            "adjacency": srk.srk_graph_layout(g), "graph_gen_s": t_gen,
            "source_in_degrees": [int(deg[s]) for s in sources]}
    print(json.dumps(line), flush=True)
    g.close()
    return 0


def run_probe(args, rank, world):
    """The random-gather ceiling itself: srk_probe_gather_ex over arrays from
    16 KB (L1-resident) to 4 GB (HBM) with each PTX cache operator; one line
    of loads/s per (size, operator)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as srk
    ops = {"default": srk.SRK_PROBE_DEFAULT, "cg": srk.SRK_PROBE_CG,
           "nc": srk.SRK_PROBE_NC, "ca": srk.SRK_PROBE_CA}
    sizes_mb = [0.015625, 0.25, 4, 16, 64, 96, 128, 256, 1024, 4096]
    table = {}
    for mb in sizes_mb:
        words = int(mb * (1 << 20)) // 4
        rates = gather_probe(srk, torch, dev, words, tuple(ops.values()))
        table["%g MB" % mb] = dict(zip(ops.keys(), rates))
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    line = {"metric": "random 4-byte gather loads/s by array size and cache operator",
            "workload": "gather_probe_sweep", "unit": "loads/s", "sms": sm,
            "value": table["64 MB"]["default"], "higher_is_better": True,
            "table": table, "note": "full-occupancy grid, 4 independent loads per thread "
                                    "per round, LCG indices; best of 2 timed runs"}
    print(json.dumps(line), flush=True)
    return 0


def run_linear(args, rank, world):
    """Linearised single-source SimRank, forward + adjoint backward: R-MAT
    scale 18, edge factor 16, lognormal(0, 0.5) FP32 weights, L = 10, c = 0.6,
    D = (1-c)I, loss = sum_v w_v s(s, v) with w ~ N(0, 1); one step = one
    forward and one backward for the next source of a uniform list."""
    import torch
    from srk_inputs import rmat_in_csr, lognormal_weights, uniform_sources
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as srk
    rp, col = rmat_in_csr(18, seed=GRAPH_SEED)
    n, m = rp.size - 1, col.size
    w = torch.from_numpy(lognormal_weights(m, seed=4)).to(dev)
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
    deg = np.diff(rp)
    srcs = [int(x) for x in uniform_sources(n, 64, seed=SOURCE_SEED) if deg[x] > 0]
    lw = torch.from_numpy(np.random.default_rng(5).normal(size=n).astype(np.float32)).to(dev)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    gw = torch.empty(m, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    L = 10

    def step(i):
        ctx = srk.srk_linear_fwd(g, w, srcs[i % len(srcs)], C, L, out)
        ev[1].record()
        srk.srk_linear_bwd(ctx, lw, gw)
        return ctx

    for i in range(args.warmup):
        step(i).free()
    fwd_ms, bwd_ms = [], []
    for i in range(args.steps):
        ev[0].record()
        ctx = step(i)
        ev[2].record()
        ev[2].synchronize()
        fwd_ms.append(ev[0].elapsed_time(ev[1]))
        bwd_ms.append(ev[1].elapsed_time(ev[2]))
        ctx.free()
    t = (np.sum(fwd_ms) + np.sum(bwd_ms)) / 1e3
    # bytes streamed: forward 2L sparse passes (P^t e_s, partial sums) over the
    # in-CSR (col 4 B + P 4 B + row 4 B per edge); backward 2L passes plus the
    # edge-gradient pass (2L vector reads per edge)
    per_pass = 12.0 * m
    fwd_bytes = 2 * L * per_pass
    bwd_bytes = 2 * L * per_pass + m * (8 + 4 * 2 * L)
    peak, peak_kind = load_peaks()
    achieved = (fwd_bytes + bwd_bytes) * args.steps / t / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "forward+backward (all kernels; the k_seg gathers are about two "
                          "thirds of device time in the launch list)",
                "peak_kind": peak_kind + " (HBM copy)",
                "bytes_per_unit": fwd_bytes + bwd_bytes, "unit_name": "forward+backward"}
    base = None
    if not args.no_cpu_baseline:
        from oracle import linear
        import torch as _t
        w64 = w.cpu().numpy().astype(np.float64)
        g64 = lw.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        reps = 0
        while reps < 1 or (time.perf_counter() - t0 < args.cpu_seconds / 2 and reps < 3):
            linear.grad(rp, col, w64, n, srcs[reps % len(srcs)], C, L, g64)
            reps += 1
        dt = (time.perf_counter() - t0) / reps
        base = {"value": 1.0 / dt, "unit": "fwd+bwd/s", "cores": _t.get_num_threads(),
                "kind": "oracle",
                "sample": "%d full forward+backward passes of the oracle (FP64 sparse "
                          "products and reverse mode)" % reps}
    line = {"metric": "linearised SimRank forward+backward per second (R-MAT 18, L=10)",
            "workload": "linear_rmat18_L10_lognormal_weights", "value": args.steps / t,
            "unit": "fwd+bwd/s", "higher_is_better": True, "n": n, "m": m,
            "fwd_ms": float(np.mean(fwd_ms)), "bwd_ms": float(np.mean(bwd_ms)),
            "fwd_GBps_streamed": fwd_bytes / (np.mean(fwd_ms) / 1e3) / 1e9,
            "bwd_GBps_streamed": bwd_bytes / (np.mean(bwd_ms) / 1e3) / 1e9,
            "dtype": "f32", "steps": args.steps, "warmup": args.warmup,
            "roofline": roofline, "cpu_baseline": base}
    print(json.dumps(line), flush=True)
    g.close()
    return 0


def run_serve(args, rank, world):
    """Serving: three resident R-MAT graphs (scales 16, 20, 23, edge factor
    16); single-source requests arrive Poisson at --rate per second for
    --serve-seconds; each picks a graph uniformly, eps uniformly from
    {0.05, 0.02, 0.01} and a source uniformly; the server admits a request
    when its device memory fits in --serve-budget-mb and sheds it otherwise.
    Reports admitted queries/s and p50/p99 latency (submission to scores on
    the host), beside the same admitted requests run one at a time."""
    import torch
    from srk_inputs import rmat_in_csr, rmat_in_csr_torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as srk
    graphs, sizes, hosts = [], [], []
    for scale in (16, 20, 23):
        if scale <= 20:
            rp, col = rmat_in_csr(scale, seed=GRAPH_SEED)
            rp_d, col_d = torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev)
        else:
            rp_d, col_d = rmat_in_csr_torch(scale, seed=GRAPH_SEED, device=dev)
        graphs.append(srk.srk_graph_load(rp_d, col_d, layout=args.layout))
        sizes.append(int(rp_d.numel()) - 1)
        hosts.append((rp_d, col_d))
    rng = np.random.default_rng(4)
    horizon = args.serve_seconds
    t_arr = np.cumsum(rng.exponential(1.0 / args.rate, size=int(args.rate * horizon * 1.2) + 16))
    t_arr = t_arr[t_arr < horizon]
    reqs = []
    for _ in range(t_arr.size):
        gi = int(rng.integers(0, 3))
        reqs.append((gi, int(rng.integers(0, sizes[gi])), float(rng.choice([0.05, 0.02, 0.01]))))
    budget = int(args.serve_budget_mb) << 20
    # warm-up (module load, pools, first launches) outside the measured run
    for gi in range(3):
        out = torch.empty(sizes[gi], dtype=torch.float64, device=dev)
        srk.srk_single_source(graphs[gi], 0, C, 0.05, 1, out)
    torch.cuda.synchronize()
    admitted = []
    with srk.srk_server_create(graphs, budget, args.serve_workers,
                               args.serve_target_ms) as srv:
        t0 = time.perf_counter()
        for k, (gi, s, eps) in enumerate(reqs):
            while time.perf_counter() - t0 < t_arr[k]:
                pass
            if srk.srk_server_submit(srv, gi, s, C, eps, QUERY_SEED + k):
                admitted.append(k)
        t_submit_end = time.perf_counter() - t0
        srk.srk_server_drain(srv)
        st = srk.srk_server_stats(srv)
    # the admitted requests again, one at a time (the plain path)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for n in sizes]
    t_plain = 0.0
    for k in admitted:
        gi, s, eps = reqs[k]
        ev[0].record()
        srk.srk_single_source(graphs[gi], s, C, eps, QUERY_SEED + k, outs[gi])
        ev[1].record()
        ev[1].synchronize()
        t_plain += ev[0].elapsed_time(ev[1]) / 1e3
    peak, peak_kind = load_peaks()
    achieved = st.target_steps * BYTES_PER_STEP / st.wall_s / 1e9 if st.wall_s else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_target_walks",
                "peak_kind": peak_kind + " (HBM copy)", "bytes_per_unit": BYTES_PER_STEP,
                "unit_name": "target-walk step",
                "note": "over the serving run's wall time (includes idle gaps)"}
    base = None
    if not args.no_cpu_baseline and admitted:
        mix = [reqs[k] for k in admitted[:6]]
        need = sorted({gi for gi, _, _ in mix})
        graphs_np = [None] * 3
        for gi in need:
            graphs_np[gi] = (hosts[gi][0].cpu().numpy(), hosts[gi][1].cpu().numpy())
        base = cpu_baseline_mix(graphs_np, mix, args.cpu_seconds)
    line = {"metric": "served single-source SimRank queries/s and latency (R-MAT 16/20/23)",
            "workload": "serve_rmat16_20_23_poisson", "value": st.queries_per_s,
            "unit": "queries/s", "higher_is_better": True,
            "offered_per_s": args.rate, "seconds": horizon, "submitted": st.submitted,
            "admitted": st.admitted, "shed": st.shed, "shed_fraction": st.shed / max(1, st.submitted),
            "completed": st.completed, "failed": st.failed,
            "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms, "max_ms": st.max_ms,
            "wall_s": st.wall_s, "target_steps": st.target_steps,
            "reserved_peak_MB": st.reserved_peak / 2 ** 20, "budget_MB": args.serve_budget_mb,
            "workers": args.serve_workers, "latency_target_ms": args.serve_target_ms,
            "submit_loop_s": t_submit_end,
            "plain_one_at_a_time_queries_per_s": len(admitted) / t_plain if t_plain else None,
            "graph_nodes": sizes, "roofline": roofline, "cpu_baseline": base}
    print(json.dumps(line), flush=True)
    for g in graphs:
        g.close()
    return 0


def run_reference(args, rank, world):
    """The oracle on the host cores, on the same workload: a step is one pass
    over the 64 sources, each query on a uniform sample of targets with its
    time scaled by n / targets (the whole run stays within a few minutes)."""
    if rank != 0:
        return 0
    rp, col, sources = make_workload()
    from oracle import sampler
    n = rp.size - 1
    rng = np.random.default_rng(11)
    k = max(64, int(n * 0.0003))
    threads = os.cpu_count() or 1
    pass_s = []
    for i in range(args.warmup + args.steps):
        t_pass = 0.0
        for s in sources:
            targets = np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)
            t0 = time.perf_counter()
            sampler.run(rp, col, n, int(s), C, EPS, QUERY_SEED, targets=targets,
                        threads=threads)
            t_pass += (time.perf_counter() - t0) * n / k
        if i >= args.warmup:
            pass_s.append(t_pass)
    per_step = float(np.mean(pass_s))
    value = len(sources) / per_step
    sample = ("%d of %d uniform targets per query, every source of the 64-source list per "
              "step, times scaled by n/targets" % (k, n))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sources_per_step": len(sources),
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_split(args, rank, world):
    """One query split across ranks by target range (the owner rule of
    Section 5.5, paper_2304_04015_gb300.split): every rank loads the whole
    graph, walks the targets it owns and the score slices are all-gathered
    (NCCL); a step is one pass over the 64 sources, each query split over
    all ranks (strong scaling: the work per step is fixed)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    else:
        pg = None
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as srk
    from paper_2304_04015_gb300.split import owner_range, split_query
    rp, col, sources = make_workload()
    n = rp.size - 1
    g = srk.srk_graph_load(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                           layout=args.layout)
    for _ in range(args.warmup):
        for s in sources:
            split_query(g, int(s), C, EPS, QUERY_SEED, rank, world)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.steps):
        for s in sources:
            full = split_query(g, int(s), C, EPS, QUERY_SEED, rank, world)
    ev[1].record()
    ev[1].synchronize()
    t = max_over_ranks(ev[0].elapsed_time(ev[1]) / 1e3, pg, dev)
    b, e = owner_range(n, rank, world)
    line = {"metric": "single-source SimRank queries/s at eps=0.02, one query split over "
                      "ranks by target range", "value": args.steps * len(sources) / t,
            "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD + "_target_split",
                       "targets_of_rank0": [b, e], "gather": "one all_gather of FP64 slices",
                       "l2": "not flushed between queries"},
            "last_score_sum": float(full.sum())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if pg:
        pg.destroy_process_group()
    return 0


def adjacency_bytes(layout: str, n: int, m: int) -> int:
    """Bytes of the adjacency the walk steps read, by layout: 4-byte entries
    (plus the hub table, a few KB to MB), 8-byte entries at n + m positions,
    or the CSR itself."""
    return {"narrow": 4 * m, "wide": 8 * (n + m), "csr": 4 * (n + 1) + 4 * m}[layout]


def source_list(n: int, rank: int):
    """The 64 sources of one rank: rank 0 takes the workload's list (seed 2);
    rank r > 0 draws its own 64 from seed 2 + 1000 r, so every rank runs a
    full list per step (weak scaling)."""
    from srk_inputs import uniform_sources
    return uniform_sources(n, N_SOURCES, seed=SOURCE_SEED + 1000 * rank)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world) if rank == 0 else 0
    if args.workload == "linear":
        return run_linear(args, rank, world) if rank == 0 else 0
    if args.workload == "serve":
        return run_serve(args, rank, world) if rank == 0 else 0
    if args.workload == "probe":
        return run_probe(args, rank, world) if rank == 0 else 0
    if args.workload == "split":
        return run_split(args, rank, world)

    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_04015_gb300 as srk

    t_gen = time.perf_counter()
    rp, col, _ = make_workload()
    t_gen = time.perf_counter() - t_gen
    n, m = rp.size - 1, col.size
    my_sources = [int(x) for x in source_list(n, rank)]
    deg = np.diff(rp)
    n_src = len(my_sources)

    rp_d = torch.from_numpy(rp).to(dev)
    col_d = torch.from_numpy(col).to(dev)
    g = srk.srk_graph_load(rp_d, col_d, layout=args.layout)
    layout = srk.srk_graph_layout(g)
    stream = torch.cuda.current_stream(dev)
    scores = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev_q = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev_k = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for e in ev_q + ev_k:
        e.record(stream)   # creates the CUDA events
    torch.cuda.synchronize()

    def query(s, out, timing=None, stats=None):
        srk.srk_single_source(g, s, C, EPS, QUERY_SEED, out, stats=stats,
                              timing_events=timing, stream=stream,
                              literal_shuffle=args.literal_shuffle,
                              warmup_rule=args.warmup_rule)

    # warm-up: W passes over the source list
    for _ in range(args.warmup):
        for s in my_sources:
            query(s, scores)
    torch.cuda.synchronize()

    # per-source step counts (one untimed pass; the counters need a sync;
    # every pass repeats the same queries, so the counts are per pass)
    stats_steps = []
    for s in my_sources:
        st = srk.SrkStats()
        query(s, scores, stats=st)
        stats_steps.append((st.target_steps, st.source_steps, st.n_walks, st.n_active_pairs,
                            st.z, st.L))
    torch.cuda.synchronize()

    # timed: K passes; each query bracketed by events on its stream, the L2
    # flush between queries outside the intervals
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    q_ms, k_ms = [], []
    t_wall = time.perf_counter()
    for step in range(args.steps):
        for i, s in enumerate(my_sources):
            flush.fill_((step * n_src + i) & 0xFF)   # evict the graph from L2 between queries
            ev_q[0].record(stream)
            query(s, scores, timing=ev_k)
            ev_q[1].record(stream)
            ev_q[1].synchronize()
            q_ms.append(ev_q[0].elapsed_time(ev_q[1]))
            k_ms.append(ev_k[0].elapsed_time(ev_k[1]))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if pg:
        pg.barrier()
    clk = clocks.stop()

    total_ms = max_over_ranks(float(np.sum(q_ms)), pg, dev)
    queries = args.steps * n_src * world
    value = queries / (total_ms / 1e3)
    tgt_steps = args.steps * sum(x[0] for x in stats_steps)
    src_steps = args.steps * sum(x[1] for x in stats_steps)
    steps_per_s = (tgt_steps + src_steps) * world / (total_ms / 1e3)

    # e2e: the same K passes through the C ABI with host output buffers
    e2e = None
    if not args.skip_e2e:
        host_scores = torch.empty(n, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        e2e_s = 0.0
        for step in range(args.steps):
            for i, s in enumerate(my_sources):
                flush.fill_((step * n_src + i) & 0xFF)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                query(s, host_scores.numpy())     # D2H copy + sync inside the call
                e2e_s += time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, pg, dev)
        e2e = {"value": queries / e2e_s, "unit": "queries/s",
               "h2d_bytes_per_step": 3108 * n_src,
               "d2h_bytes_per_step": 8 * n * n_src,
               "note": "graph resident (loaded once); per query the host passes "
                       "(s, c, eps, seed) and the 3108-byte sample-count table as "
                       "kernel arguments and reads back n FP64 scores; a step is "
                       "%d queries" % n_src}

    peak_hbm, peak_kind = load_peaks()
    kern_s = float(np.sum(k_ms)) / 1e3
    target_steps_per_s = tgt_steps / kern_s
    hbm_achieved = tgt_steps * BYTES_PER_STEP / kern_s / 1e9
    per_step = recorded_traffic()
    launches = args.steps * n_src
    traffic = per_step * tgt_steps / launches if per_step is not None else None
    adj_b = adjacency_bytes(layout, n, m)
    l2_b = torch.cuda.get_device_properties(dev).L2_cache_size
    gather = None
    l2_rate = None
    if not args.skip_probe:
        ops = (srk.SRK_PROBE_DEFAULT, srk.SRK_PROBE_CG, srk.SRK_PROBE_NC, srk.SRK_PROBE_CA)
        by_op = gather_probe(srk, torch, dev, adj_b // 4, ops)     # graph-sized array
        l2_rate = by_op[0]
        hbm_rate = gather_probe(srk, torch, dev, 1 << 30)[0]       # 4 GB array
        l1_rate = gather_probe(srk, torch, dev, 1 << 12)[0]        # 16 KB array (L1 hits)
        gather = {"probe_gathers_per_s_graph_sized": l2_rate,
                  "probe_gathers_per_s_4GB": hbm_rate,
                  "probe_gathers_per_s_16KB": l1_rate,
                  "probe_graph_sized_by_cache_op": dict(zip(("default", "cg", "nc", "ca"),
                                                            by_op)),
                  "kernel_steps_per_s": target_steps_per_s,
                  "frac_of_graph_sized_probe": target_steps_per_s / l2_rate,
                  "note": "one scattered 4-byte adjacency read per target-walk step; "
                          "probe = srk_probe_gather, independent random loads at full "
                          "occupancy on an array the size of the adjacency"}
    fits_l2 = adj_b <= l2_b
    hbm_frac = hbm_achieved / peak_hbm
    common = {"kernel": "k_target_walks", "traffic": traffic,
              "traffic_unit": "DRAM bytes per launch (ncu, recorded for these kernel sources)",
              "kernel_ms_per_launch": float(np.mean(k_ms)),
              "kernel_share_of_query": float(np.sum(k_ms) / np.sum(q_ms)),
              "adjacency_bytes": adj_b, "l2_bytes": l2_b,
              "hbm_copy": {"achieved": hbm_achieved, "peak": peak_hbm, "unit": "GB/s",
                           "frac": hbm_frac, "peak_kind": peak_kind + " (HBM copy)",
                           "bytes_per_unit": BYTES_PER_STEP,
                           "unit_name": "target-walk step (row_ptr pair + one entry)"}}
    if l2_rate is not None:
        roofline = {"bound": "l2_gather" if fits_l2 else "hbm_gather",
                    "achieved": target_steps_per_s / 1e9, "peak": l2_rate / 1e9,
                    "unit": "Gloads/s", "frac": target_steps_per_s / l2_rate,
                    "peak_kind": "measured live: random 4-byte gather probe on an array the "
                                 "size of the adjacency (%d MB)" % (adj_b >> 20),
                    "unit_name": "target-walk step (one dependent scattered adjacency load)",
                    **common}
        sps = recorded_l2_sectors()
        if sps is not None:
            # each probe load misses L1 and takes one L2 sector; a step of the
            # kernel takes fewer (some of its loads hit L1)
            roofline["l2_sectors"] = {
                "per_step": sps, "achieved": target_steps_per_s * sps / 1e9,
                "peak": l2_rate / 1e9, "unit": "Gsectors/s",
                "frac": target_steps_per_s * sps / l2_rate,
                "source": "L2 sectors requested by L1 per step from the recorded ncu "
                          "capture of these kernel sources"}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": peak_hbm,
                    "unit": "GB/s", "frac": hbm_frac,
                    "peak_kind": peak_kind + " (HBM copy)",
                    "bytes_per_unit": BYTES_PER_STEP, "unit_name": "target-walk step",
                    **common}

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(rp, col, my_sources, args.cpu_seconds,
                            literal_shuffle=args.literal_shuffle, warmup_rule=args.warmup_rule)

    zero_src = [s for s in my_sources if deg[s] == 0]
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD + variant_suffix(args),
                       "variant": variant_name(args),
                       "graph": "R-MAT scale 20, edge factor 16, "
                       "(0.57,0.19,0.19,0.05), dedup, no self-loops, seed %d" % GRAPH_SEED,
                       "n": n, "m": m, "c": C, "eps": EPS,
                       "step": "one pass over all %d sources of the list, one query per "
                               "launch" % n_src,
                       "sources_per_step": n_src,
                       "queries_timed_per_rank": args.steps * n_src,
                       "sources_timed": my_sources,
                       "sources_without_in_neighbours": len(zero_src),
                       "source_seed": SOURCE_SEED, "query_seed": QUERY_SEED,
                       "adjacency": layout,
                       "z": stats_steps[0][4], "N_tot": stats_steps[0][2],
                       "L": int(stats_steps[0][5]),
                       "l2": "256 MB buffer written between queries (outside the timed intervals)",
                       "timing": "sum of per-query CUDA-event intervals on the query stream",
                       "parallelism": "each rank runs its own 64-source list" if world > 1
                       else "1 GPU"},
            "walk_steps_per_s": steps_per_s,
            "target_steps_per_query": tgt_steps / launches,
            "query_ms": {"best": float(np.min(q_ms)), "median": float(np.median(q_ms)),
                         "max": float(np.max(q_ms)),
                         "note": "per-query CUDA-event times on this rank; sources differ "
                                 "in work (active pairs per target); a source without "
                                 "in-neighbours returns after the source phases"},
            "roofline": roofline, "gather_roofline": gather, "cpu_baseline": base,
            "e2e": e2e, "clocks": clk,
            "gpu_launches": 9 * launches,
            "wall_s_timed_loop": t_wall, "graph_gen_s": t_gen}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
