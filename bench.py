#!/usr/bin/env python3
"""Benchmark of the colour-coding hot path on one GB300 (or N replicas).

Workload: Chung-Lu power-law graph, n = 1M, m ~ 10M, degree exponent 2.5,
largest expected degree 10k (synthetic, seeded); k = 5 colours, 64-bit
counts.  One step = colour the graph, build the exact count tables for
h = 1..5 (neighbour sums + merges), prefix the level totals, draw 1M uniform
colourful 5-treelets, classify their induced 5-graphlets and estimate the
21 graphlet counts -- every step of the path, through the C ABI.

value: DP table entries (n x live entries per node) per second of step time.
Also reported: samples/s, per-phase and per-kernel device times, the
roofline of the dominant kernel, an end-to-end number through host buffers,
the CPU oracle as a baseline, and SM clocks sampled during the timed region.

Multi-GPU: one process per GPU (torchrun); every rank builds and samples its
own colouring of the same graph (independent replicas, no data-path
collective), so per-GPU work is fixed as N grows ("weak").  --impl reference
times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

K = 5
BITS = 64
SAMPLES = 1_000_000
R_H = [0, 1, 1, 2, 4, 9, 20, 48, 115]  # rooted shapes per size


def workload_graph(small: bool):
    if small:
        return synth.er_1k(), "er_1k"
    return synth.chung_lu_1m(), "chung_lu_1m_k5"


def workload_config(graph, wname: str, k: int, samples: int, args, world: int) -> dict:
    """The `config` of the default workload's JSON line (both arms)."""
    return {"workload": wname, "n": int(graph.n), "m": int(graph.nnz) // 2, "k": k, "count_bits": BITS,
            "samples_per_step": samples, "zero_root": bool(args.zero_root),
            "skip_round": bool(args.skip_round),
            "star_samples_per_step": samples if args.skip_round else 0,
            "l2": "flushed between steps (256 MiB write, outside the per-step events)",
            "parallelism": f"replicas{world}"}


def live_entries_per_node(k: int) -> int:
    return sum(R_H[h] * math.comb(k - 1, h - 1) for h in range(1, k + 1))


def geometry(k: int):
    Bc = {h: math.comb(k - 1, h - 1) for h in range(1, k + 1)}
    Bs = {h: math.comb(k - 1, h) for h in range(1, k)}
    Wc = {h: R_H[h] * Bc[h] for h in Bc}
    Ws = {h: R_H[h] * Bs[h] for h in Bs}
    return Wc, Ws


def algorithmic_bytes(name: str, n: int, nnz: int, k: int, B: int):
    """Compulsory DRAM bytes of one launch of a build kernel (each input row
    read once, each output row written once, plus the CSR it walks)."""
    Wc, Ws = geometry(k)
    csr = 8 * (n + 1) + 4 * nnz + n
    if name == "gather_h1":
        return csr + n * (k - 1) * B
    if name.startswith("gather_h"):
        h = int(name[len("gather_h"):])
        return n * Wc[h] * B + n * Ws[h] * B + csr
    if name.startswith("merge_h"):
        import paper_2009_03052_gb300 as M
        h = int(name[len("merge_h"):])
        used1, used2 = set(), set()
        for code in M.shape_info(h)["code"]:
            # s_T of the shape; T'' is the subtree of the first root child
            bits = format(int(code), "0%db" % (2 * (h - 1)))
            depth, end = 0, 0
            for i, ch in enumerate(bits):
                depth += 1 if ch == "1" else -1
                if depth == 0:
                    end = i + 1
                    break
            h2 = end // 2
            used1.add(h - h2)
            used2.add(h2)
        rd = sum(Wc[x] for x in used1 if x > 1) + sum(Ws[x] for x in used2)
        return n * (rd + Wc[h]) * B
    return None


# ---------------------------------------------------------------------------
# combining ranks
# ---------------------------------------------------------------------------
def job_throughput(units_per_rank: float, my_ms: float, world: int, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: every rank processed
    units_per_rank in my_ms; the job took the slowest rank's time.  Returns
    (max ms over ranks, units of all ranks per second)."""
    if world > 1:
        import torch
        t = torch.tensor([my_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        my_ms = float(t.item())
    return my_ms, units_per_rank * world / (my_ms / 1e3)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "10", "-i", str(self.device)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts once nvidia-smi is sampling (at most 3 s)
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle baseline
# ---------------------------------------------------------------------------
def oracle_step_rate(graph, k: int, n_samples: int, seed: int, threads: int):
    """Time the oracle on one bounded step of the workload, as run (nothing
    extrapolated): its table build on the full graph, then n_samples uniform
    samples with classification and estimates.  Returns the step's DP-table
    entries per second of step time, and the build and sampling rates."""
    import oracle
    oracle.build()
    oracle.class_codes(k)  # class list precomputed outside the timing
    oracle.sigma(k)
    colors = oracle.color(graph.n, k, seed)
    t0 = time.perf_counter()
    T = oracle.Tables(graph, colors, k, BITS, nthreads=threads)
    t1 = time.perf_counter()
    T.estimate_uniform(k, seed=seed, n_samples=n_samples)
    t2 = time.perf_counter()
    build_s, samp_s = t1 - t0, t2 - t1
    entries = graph.n * live_entries_per_node(k)
    return {"value": entries / (build_s + samp_s), "build_s": build_s, "sample_s": samp_s,
            "step_s": build_s + samp_s, "build_entries_per_s": entries / build_s,
            "samples_per_s": n_samples / samp_s}


ORACLE_STEP_SAMPLES = 2000  # samples in one bounded oracle step (about 0.5 s of its sampling)


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    graph, wname = workload_graph(args.small)
    threads = os.cpu_count() or 1
    k = K if not args.small else 4
    n_samp = ORACLE_STEP_SAMPLES if not args.small else 10_000
    # warm-up: the oracle on a small graph of the same family
    warm = synth.chung_lu_scaled(5000, seed=1)
    for i in range(args.warmup):
        oracle_step_rate(warm, K, 100, 100 + i, threads)
    res = [oracle_step_rate(graph, k, n_samp, 10 + i, threads) for i in range(args.steps)]
    step_s = sum(r["step_s"] for r in res)
    entries = graph.n * live_entries_per_node(k)
    val = entries * args.steps / step_s
    sample = (f"one step = the oracle's build of the full {wname} graph plus {n_samp} uniform samples "
              f"with classification and estimates, as run (the GPU step draws "
              f"{SAMPLES if not args.small else 10_000})")
    line = {
        "impl": "reference", "metric": "DP table entries/s", "value": val,
        "unit": "entries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(graph, wname, k, SAMPLES if not args.small else 10_000, args, world),
        "cpu_baseline": {"value": val, "unit": "entries/s", "cores": threads, "kind": "oracle",
                         "sample": sample,
                         "build_entries_per_s": statistics.median(r["build_entries_per_s"] for r in res),
                         "samples_per_s": statistics.median(r["samples_per_s"] for r in res)},
        "e2e": {"value": val, "unit": "entries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist

    import paper_2009_03052_gb300 as M

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    M.build()
    M.load()
    graph, wname = workload_graph(args.small)
    k = 4 if args.small else K
    samples = 10_000 if args.small else SAMPLES
    n, nnz = graph.n, graph.nnz
    G = M.Graph.from_csr(graph)
    colbuf = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    phase = {"build": [], "sample": []}

    def step(seed: int, record: bool):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        col = M.color(G, k, seed, out=colbuf)
        T = M.Tables(G, col, k, BITS, zero_root=args.zero_root, skip_round=args.skip_round)
        e1.record(stream)
        est, hits, _ = T.estimate(k, seed=seed, samples=samples,
                                  star_samples=samples if args.skip_round else 0)
        e2.record(stream)
        T.free()
        if record:
            e2.synchronize()
            phase["build"].append(e0.elapsed_time(e1))
            phase["sample"].append(e1.elapsed_time(e2))
        return hits

    seed0 = 1000 * rank
    for i in range(args.warmup):
        step(seed0 + i, False)
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (126 MB)

    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    M.profile_reset()
    M.profile_enable(True)
    launches0 = M.launch_count()
    step_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)  # evict L2 between steps, outside the step's events
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(seed0 + args.warmup + i, True)
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    launches = M.launch_count() - launches0
    prof = {k: v[:2] for k, v in M.profile_read().items() if v[1] > 0}
    clk = clocks.stop()
    # the bytes each kernel counts, from the last timed step run once more
    # with counting on (its own instantiation; samples are deterministic)
    M.profile_reset()
    M.profile_enable(True, count_bytes=True)
    step(seed0 + args.warmup + args.steps - 1, False)
    torch.cuda.synchronize()
    counted = M.profile_read(with_bytes=True)
    M.profile_enable(False)
    if world > 1:
        dist.barrier()
    entries = n * live_entries_per_node(k)
    if args.skip_round:  # level k-1 is never built
        entries -= n * R_H[k - 1] * math.comb(k - 1, k - 2)
    if args.zero_root:  # level k is built at colour-0 nodes only
        n0 = int((M.color(G, k, seed0, out=colbuf) == 0).sum().item())
        entries -= (n - n0) * R_H[k]
    total_ms, value = job_throughput(entries * args.steps, sum(step_ms), world, dist, "cuda")
    ms_per_step = total_ms / args.steps
    build_ms = statistics.mean(phase["build"])
    sample_ms = statistics.mean(phase["sample"])

    # the schedules the autotuner chose for this workload's levels
    gn, gnnz, gmaxd = G.info()
    schedules = {}
    for h in range(2, k + 1):
        schedules[f"merge_h{h}"] = M.autotune_choice(1, k, BITS, h, gn, gnnz, gmaxd)
        if h < k:
            schedules[f"gather_h{h}"] = M.autotune_choice(0, k, BITS, h, gn, gnnz, gmaxd)

    # per-kernel shares and the roofline of the dominant kernel
    ktot = sum(v[0] for v in prof.values()) or 1.0
    kernels = {name: {"ms": round(ms, 4), "launches": cnt, "share": round(ms / ktot, 4)}
               for name, (ms, cnt) in sorted(prof.items(), key=lambda x: -x[1][0])}
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peaks = json.load(open(peaks_path))
        hbm_peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        hbm_peak, peak_src = 6800.0, "fallback"
    def roofline(nm):
        ms, cnt = prof[nm]
        item = None
        cms, ccnt, citems = counted.get(nm, (0.0, 0, 0))
        sectors = counted.get(nm + " sectors", (0.0, 0, 0))[2]
        if sectors > 0 and ccnt > 0:
            # the sector model of the sampler's bytes (32 B per random access:
            # root-search probes, each scanned neighbour's row entry, chunk-
            # and adjacency-search probes; contiguous runs by their bytes),
            # per launch of the counting step
            by = sectors / ccnt
            src = ("counted by the kernel, 32-byte sector model: 32 B per random access, "
                   "contiguous runs by their bytes (one extra counted step)")
            item = int(citems / ccnt)
        else:
            by = algorithmic_bytes(nm, n, nnz, k, BITS // 8)
            src = "compulsory bytes (each row read once, written once, plus the CSR)"
        if by is None:
            return None
        achieved = by / (ms / cnt / 1e3) / 1e9
        traffic = traffic_of(wname, nm, schedules.get(nm))
        out = {"kernel": nm, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
               "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
               "traffic": traffic, "algorithmic_bytes": int(by),
               "bytes_model": src, "peak_source": peak_src, "avg_launch_ms": round(ms / cnt, 4)}
        if item is not None:  # the bytes of the data items themselves
            out["item_bytes"] = item
            out["item_frac"] = round(item / (ms / cnt / 1e3) / 1e9 / hbm_peak, 4)
        if traffic:  # the DRAM bytes of the ncu capture over this run's launch time
            dram = traffic / (ms / cnt / 1e3) / 1e9
            out["dram_gbs"] = round(dram, 1)
            out["dram_frac"] = round(dram / hbm_peak, 4)
        return out

    top = max(prof.items(), key=lambda x: x[1][0])[0] if prof else None
    roof = roofline(top) if top else None
    build_kernels = [nm for nm in prof if nm.startswith(("gather", "merge"))]
    roof_build = roofline(max(build_kernels, key=lambda x: prof[x][0])) if build_kernels else None

    # non-zero entries of one build (what a zero-suppressed table keeps),
    # counted outside the timed steps
    Tn = M.Tables(G, M.color(G, k, seed0, out=colbuf), k, BITS, zero_root=args.zero_root,
                  skip_round=args.skip_round)
    nonzero = sum(Tn.nonzeros(h) for h in range(1, k + 1) if not (args.skip_round and h == k - 1))
    Tn.free()

    # end to end through the C ABI with host buffers: graph upload, colour,
    # build, sample, estimates copied back
    e2e_ms = []
    rp_pin = torch.from_numpy(graph.row_ptr).pin_memory()
    col_pin = torch.from_numpy(graph.col.view(np.int32)).pin_memory()
    h2d = graph.row_ptr.nbytes + graph.col.nbytes
    d2h = 0
    for i in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = M.Graph(rp_pin, col_pin, trusted=True)
        col = M.color(G2, k, seed0 + 77 + i, out=colbuf)
        T2 = M.Tables(G2, col, k, BITS, zero_root=args.zero_root, skip_round=args.skip_round)
        est, hits, _ = T2.estimate(k, seed=seed0 + 77 + i, samples=samples,
                                   star_samples=samples if args.skip_round else 0)
        d2h = est.nbytes + hits.nbytes
        T2.free()
        G2.free()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    _, e2e_value = job_throughput(entries, statistics.median(e2e_ms), world, dist, "cuda")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        n_samp = ORACLE_STEP_SAMPLES if not args.small else 10_000
        r = oracle_step_rate(graph, k, n_samp, 5, threads)
        cpu = {"value": r["value"], "unit": "entries/s", "cores": threads, "kind": "oracle",
               "sample": (f"one bounded step as run: the oracle's build of the full {wname} graph "
                          f"({r['build_s']:.2f} s) plus {n_samp} uniform samples with classification "
                          f"and estimates ({r['sample_s']:.2f} s)"),
               "build_entries_per_s": r["build_entries_per_s"], "samples_per_s": r["samples_per_s"]}


    extra = {}
    if rank == 0 and not args.no_extra and not args.small:
        del G
        torch.cuda.empty_cache()
        extra = extra_workloads(M, torch)

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": "DP table entries/s", "value": value, "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": workload_config(graph, wname, k, samples, args, world),
        "samples_per_s": samples * args.steps * world / (total_ms / 1e3),
        "phases_ms": {"build": round(build_ms, 3), "sample_classify_estimate": round(sample_ms, 3)},
        "build_entries_per_s": entries / (build_ms / 1e3),
        "nonzero_entries": int(nonzero), "nonzero_entries_per_s": nonzero / (build_ms / 1e3),
        "roofline": roof, "roofline_build": roof_build, "top_kernel": top, "kernels": kernels,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "entries/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": statistics.median(e2e_ms),
                "path": "mc_load_graph (pinned host CSR, trusted) + mc_color + mc_build_tables + "
                        "mc_estimate_counts (host estimates)"},
        "cpu_baseline": cpu, "clocks": clk, "schedules": schedules,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)


def extra_workloads(M, torch) -> dict:
    """k = 7 and k = 8 beside the k = 5 line (u128 counts): build entries/s,
    uniform and adaptive (AGS) colourful graphlet samples/s.
      k7_rmat22: R-MAT scale 22, edge factor 16 (a, b, c = .57, .19, .19);
                 10M uniform samples, AGS with cbar = 1000 and 10M samples.
      k8_cl2m:   Chung-Lu n = 2M, m ~ 20M, exponent 2.5; 1M uniform
                 8-samples, AGS with cbar = 1000 and 1M samples.
    Builds: one warm-up (it autotunes), then the median of two; L2 flushed
    before each timed call."""
    out = {}
    s = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn):
        flush.fill_(7)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        r = fn()
        b.record(s)
        b.synchronize()
        return a.elapsed_time(b), r

    for name, make, k, uni, ags in (
            ("k7_rmat22", lambda: synth.rmat(22, 16, seed=0), 7, 10_000_000, 10_000_000),
            ("k8_cl2m", lambda: synth.chung_lu(2_000_000, 20_000_000, 2.5, max_degree=10_000.0, seed=0),
             8, 1_000_000, 1_000_000)):
        g = make()
        G = M.Graph.from_csr(g, trusted=True)
        col = M.color(G, k, 11)
        M.sigma(k)
        T = M.Tables(G, col, k, 128)  # warm-up build (autotunes)
        T.free()
        bms = []
        for _ in range(2):
            ms, T = timed(lambda: M.Tables(G, col, k, 128))
            bms.append(ms)
            if _ == 0:
                T.free()
        T.total(k)
        for j in range(M.num_unrooted(k)):
            T.total(k, j)
        T.estimate(k, seed=1, samples=100_000)  # warm-up of the samplers
        T.estimate(k, seed=1, samples=100_000, mode=M.MC_EST_AGS, cbar=1000)
        ums, _ = timed(lambda: T.estimate(k, seed=2, samples=uni))
        ams, (_, _, st) = timed(lambda: T.estimate(k, seed=3, samples=ags, mode=M.MC_EST_AGS, cbar=1000))
        T.free()
        packed = {}
        if k == 7:
            # the same tables zero-suppressed (Section 3.2.1), with the
            # table's width or each row's own width (Section 3.3.3)
            for pname, vl in (("succinct", False), ("varlen", True)):
                pms, P = timed(lambda: M.Tables(G, col, k, 128, succinct=True, varlen=vl))
                dense_b, stored_b = P.table_bytes()
                P.estimate(k, seed=1, samples=100_000)
                pums, _ = timed(lambda: P.estimate(k, seed=2, samples=1_000_000))
                packed[pname] = {"build_ms": round(pms, 3), "dense_bytes": dense_b, "stored_bytes": stored_b,
                                 "stored_over_dense": round(stored_b / dense_b, 4),
                                 "uniform_samples_per_s": 1_000_000 / (pums / 1e3)}
                P.free()
        entries = g.n * live_entries_per_node(k)
        bm = statistics.median(bms)
        out[name] = {"n": g.n, "m": g.m, "k": k, "count_bits": 128, "build_ms": round(bm, 3),
                     "build_entries_per_s": entries / (bm / 1e3),
                     "uniform_samples": uni, "uniform_samples_per_s": uni / (ums / 1e3),
                     "ags_samples": st["samples"], "ags_samples_per_s": st["samples"] / (ams / 1e3),
                     "ags_switches": st["switches"], "ags_over_uniform_speed": (st["samples"] / ams) / (uni / ums)}
        out[name].update(packed)
        del G
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# batching: many colourings of one graph plus many uneven graphs, one build
# ---------------------------------------------------------------------------
def batch_instances():
    """64 colourings of a Chung-Lu graph (n=200k, m=2M, exponent 2.3) plus 32
    Erdos-Renyi / Chung-Lu graphs (n log-uniform in [1k, 100k], average
    degree uniform in [4, 20], seed = index)."""
    base = synth.chung_lu(200_000, 2_000_000, 2.3, seed=0)
    rng = np.random.default_rng(7)
    extra = []
    for i in range(32):
        n = int(np.exp(rng.uniform(np.log(1_000), np.log(100_000))))
        deg = float(rng.uniform(4, 20))
        extra.append(synth.erdos_renyi(n, deg, seed=i) if i % 2 == 0
                     else synth.chung_lu(n, int(n * deg / 2), 2.3, seed=i))
    return [base] * 64 + extra


def run_batch(args):
    import torch
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    k, bits = 6, 128
    graphs = batch_instances()
    G = {}
    for g in graphs:
        if id(g) not in G:
            G[id(g)] = M.Graph.from_csr(g)
    gl = [G[id(g)] for g in graphs]
    cols = [M.color(gi, k, 1000 + i, out=torch.empty(gi.n, dtype=torch.uint8, device="cuda"))
            for i, gi in enumerate(gl)]
    entries = sum(g.n for g in graphs) * live_entries_per_node(k)
    s = torch.cuda.current_stream()

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        out = fn()
        b.record(s)
        b.synchronize()
        return a.elapsed_time(b), out

    def batched():
        T, offs = M.Tables.batch(gl, cols, k, bits)
        T.free()

    def single():
        for gi, c in zip(gl, cols):
            M.Tables(gi, c, k, bits).free()

    for _ in range(args.warmup):
        batched()
        single()
    bms = [timed(batched)[0] for _ in range(args.steps)]
    sms = [timed(single)[0] for _ in range(args.steps)]
    bm, sm = statistics.median(bms), statistics.median(sms)

    # the whole batch as one captured CUDA graph: the union tables built
    # once, then per step the 96 colourings copied into the union's colour
    # buffer and an in-place rebuild of every instance replayed
    TU, offs = M.Tables.batch(gl, cols, k, bits)
    ubuf = torch.empty(int(offs[-1]), dtype=torch.uint8, device="cuda")
    ucols = torch.cat(cols)
    side0 = torch.cuda.Stream()
    side0.wait_stream(s)
    with torch.cuda.stream(side0):
        ubuf.copy_(ucols)
        TU.rebuild(ubuf)
    s.wait_stream(side0)
    TU.status()
    ugraph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(ugraph):
        TU.rebuild(ubuf)

    def union_replay():
        ubuf.copy_(ucols)
        ugraph.replay()

    for _ in range(args.warmup):
        union_replay()
    ums = statistics.median(timed(union_replay)[0] for _ in range(args.steps))
    TU.status()
    TU.free()

    # the 64 colourings of the shared graph: one in-place rebuild captured
    # into a CUDA graph and replayed per colouring, against a fresh build each
    g0 = gl[0]
    buf = cols[0].clone()
    T0 = M.Tables(g0, buf, k, bits)
    side = torch.cuda.Stream()
    side.wait_stream(s)
    with torch.cuda.stream(side):
        T0.rebuild(buf)
    s.wait_stream(side)
    T0.status()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        T0.rebuild(buf)

    def replay64():
        for c in cols[:64]:
            buf.copy_(c)
            graph.replay()

    def single64():
        for c in cols[:64]:
            M.Tables(g0, c, k, bits).free()

    for _ in range(args.warmup):
        replay64()
        single64()
    rms = statistics.median(timed(replay64)[0] for _ in range(args.steps))
    s64 = statistics.median(timed(single64)[0] for _ in range(args.steps))
    T0.status()
    entries64 = 64 * g0.n * live_entries_per_node(k)
    print(json.dumps({
        "metric": "DP table entries/s", "value": entries / (bm / 1e3), "unit": "entries/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": bm,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128",
        "data": "synthetic",
        "config": {"workload": "batch_cl200k_x64_plus_32_graphs_k6", "instances": len(graphs),
                   "nodes": sum(g.n for g in graphs), "k": k, "count_bits": bits},
        "per_instance": {"value": entries / (sm / 1e3), "ms_per_step": sm,
                         "launch_path": "one mc_build_tables per instance"},
        "batched_over_per_instance": sm / bm,
        "union_rebuild_graph": {
            "ms": ums, "entries_per_s": entries / (ums / 1e3), "over_per_instance": sm / ums,
            "path": "the union of all 96 instances built once; per step the colourings copied into its "
                    "colour buffer and an in-place rebuild of every instance replayed from one captured "
                    "CUDA graph (autotuned schedules)"},
        "rebuild_graph_64_colourings": {
            "ms": rms, "entries_per_s": entries64 / (rms / 1e3), "fresh_builds_ms": s64,
            "speedup": s64 / rms,
            "path": "mc_rebuild_tables captured once into a CUDA graph, replayed per colouring "
                    "(colours copied into the captured buffer first) vs mc_build_tables per colouring"}}),
          flush=True)


# ---------------------------------------------------------------------------
# R-MAT scale 22, k = 7: build plus 10M adaptive samples
# ---------------------------------------------------------------------------
def run_rmat(args):
    import torch
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    k, bits, samples = 7, 128, 10_000_000
    g = synth.rmat(args.rmat_scale, 16, seed=0)
    G = M.Graph.from_csr(g, trusted=True)
    colbuf = torch.empty(g.n, dtype=torch.uint8, device="cuda")
    M.sigma(k)
    s = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = []
    for i in range(args.warmup + args.steps):
        flush.fill_(i & 0xFF)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(s)
        col = M.color(G, k, 500 + i, out=colbuf)
        T = M.Tables(G, col, k, bits)
        T.total(k)
        e[1].record(s)
        est, hits, st = T.estimate(k, seed=i, samples=samples, mode=M.MC_EST_AGS, cbar=1000)
        e[2].record(s)
        # uniform sampling of the same budget, for the AGS / uniform speed ratio
        eu = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        eu[0].record(s)
        T.estimate(k, seed=i, samples=samples)
        eu[1].record(s)
        eu[1].synchronize()
        T.free()
        if i >= args.warmup:
            res.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), st, eu[0].elapsed_time(eu[1])))
    build_ms = statistics.median(r[0] for r in res)
    ags_ms = statistics.median(r[1] for r in res)
    uni_ms = statistics.median(r[3] for r in res)
    entries = g.n * live_entries_per_node(k)
    st = res[-1][2]
    # per-kernel times of one more build (CUDA events of the library's profiler)
    M.profile_reset()
    M.profile_enable(True)
    T = M.Tables(G, M.color(G, k, 500, out=colbuf), k, bits)
    torch.cuda.synchronize()
    kern = {nm: round(v[0], 3) for nm, v in sorted(M.profile_read().items(), key=lambda x: -x[1][0])}
    M.profile_enable(False)
    T.free()
    print(json.dumps({
        "metric": "DP table entries/s", "value": entries / (build_ms / 1e3), "unit": "entries/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": build_ms + ags_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128",
        "data": "synthetic",
        "config": {"workload": f"rmat{args.rmat_scale}_k7_ags10m", "n": g.n, "m": g.m, "k": k,
                   "count_bits": bits,
                   "rmat": [0.57, 0.19, 0.19], "edge_factor": 16, "ags_samples": samples,
                   "cbar": 1000, "l2": "flushed between steps"},
        "build_ms": build_ms, "ags_ms": ags_ms,
        "ags_samples_per_s": st["samples"] / (ags_ms / 1e3), "ags_stats": st,
        "uniform_samples_per_s": samples / (uni_ms / 1e3),
        "ags_over_uniform_speed": (st["samples"] / ags_ms) / (samples / uni_ms),
        "build_kernels_ms": kern}), flush=True)


# ---------------------------------------------------------------------------
# serving: a Poisson stream of requests over device-resident k = 8 tables
# ---------------------------------------------------------------------------
def run_serve(args):
    import threading

    import torch
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    k, bits = 8, 128
    g = synth.chung_lu(2_000_000, 20_000_000, 2.5, max_degree=10_000.0, seed=0)
    G = M.Graph.from_csr(g, trusted=True)
    col = M.color(G, k, 1)
    t0 = time.perf_counter()
    T = M.Tables(G, col, k, bits, own_memory=True)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    for h in range(5, k + 1):  # root indices and graphlet catalogues, before the stream
        T.total(h)
        M.sigma(h)
    rng = np.random.default_rng(3)
    n_req = args.requests
    reqs = []
    for i in range(n_req):
        h = int(rng.integers(5, k + 1))
        if rng.random() < 0.1:
            reqs.append(("ags", h, 7000 + i, int(10 ** rng.uniform(5, 6))))
        else:
            reqs.append(("sample", h, 1000 + i, int(10 ** rng.uniform(3, 6))))
    gaps = rng.exponential(1.0 / args.rate, size=n_req)
    S = M.Server([T], slots=args.slots)
    ids = [None] * n_req
    done = []

    def collect():
        for i in range(n_req):
            while ids[i] is None:
                time.sleep(1e-4)
            done.append(S.wait(ids[i]))

    th = threading.Thread(target=collect)
    th.start()
    w0 = time.perf_counter()
    next_t = w0
    for i, r in enumerate(reqs):
        next_t += gaps[i]
        dt = next_t - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        if r[0] == "sample":
            ids[i] = S.submit_sample(0, r[1], r[2], r[3])
        else:
            ids[i] = S.submit_estimate(0, r[1], r[2], r[3], mode=M.MC_EST_AGS, cbar=1000)
    th.join()
    wall = time.perf_counter() - w0
    S.free()
    lat = np.array([d["latency_us"] for d in done]) / 1e3
    samples = sum(r[3] for r in reqs)
    print(json.dumps({
        "metric": "colorful graphlet samples/s (served)", "value": samples / wall,
        "unit": "samples/s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": wall * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128",
        "data": "synthetic",
        "config": {"workload": "serve_cl2m_k8", "n": g.n, "m": g.m, "k": k, "count_bits": bits,
                   "requests": n_req, "arrival_rate_per_s": args.rate, "slots": args.slots,
                   "mix": "90% sample requests (10^3-10^6 samples, h 5..8), 10% AGS (10^5-10^6)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "queue_ms_p50": float(np.percentile([d["queue_us"] / 1e3 for d in done], 50)),
        "build_s": build_s}), flush=True)


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch, from
# one ncu capture of the named kernel on the named workload (the summaries in
# profiles/), with a hash of the kernel's source file when it was captured:
# the figure is reported only while that source is unchanged.
TRAFFIC: dict = {
    # profiles/sample_kernel_chung_lu_1m_k5.md
    ("chung_lu_1m_k5", "sample"): (2_766_753_792, "ddde42efec355d4f"),
    # profiles/gather_kernel_chung_lu_1m_k5.md, under schedules 6, 4, 4
    ("chung_lu_1m_k5", "gather_h2"): (548_702_208, "887df3f50aaa2286", 6),
    ("chung_lu_1m_k5", "gather_h3"): (1_256_040_192, "887df3f50aaa2286", 4),
    ("chung_lu_1m_k5", "gather_h4"): (1_108_238_080, "887df3f50aaa2286", 4),
}
KERNEL_SOURCE = {"sample": "sample.cu", "gather": "gather.cuh", "merge": "build.cu"}


def source_hash(kernel: str) -> str:
    import hashlib
    base = kernel.split("_h")[0]
    path = os.path.join(ROOT, "paper_2009_03052_gb300", "csrc", KERNEL_SOURCE.get(base, ""))
    if not os.path.isfile(path):
        return ""
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def traffic_of(workload: str, kernel: str, schedule: int | None = None):
    """The captured DRAM bytes per launch, while the kernel's source and (if
    recorded) the autotuned schedule are those of the capture; else None."""
    entry = TRAFFIC.get((workload, kernel))
    if not entry or entry[1] != source_hash(kernel):
        return None
    if len(entry) > 2 and schedule is not None and entry[2] != schedule:
        return None
    return entry[0]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--small", action="store_true", help="the 1k-node ER case (k = 4)")
    ap.add_argument("--workload", choices=["default", "batch", "serve", "rmat"], default="default",
                    help="batch: 96 instances built in one pass vs one by one (k = 6, u128); "
                         "serve: a request stream over k = 8 tables; "
                         "rmat: R-MAT scale 22, k = 7, build + 10M adaptive samples")
    ap.add_argument("--requests", type=int, default=200, help="serve: number of requests")
    ap.add_argument("--rmat-scale", type=int, default=22, help="rmat: log2 of the node count")
    ap.add_argument("--rate", type=float, default=100.0, help="serve: arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent requests")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: skip the k = 7 (R-MAT 22) and k = 8 (Chung-Lu 2M) keys")
    ap.add_argument("--zero-root", action="store_true",
                    help="store level k at colour-0 nodes only (Section 3.4.1)")
    ap.add_argument("--skip-round", action="store_true",
                    help="round skipping: level k from balanced decompositions, level k-1 not "
                         "built, k-stars sampled uncoloured (as many as table samples)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "rmat":
        run_rmat(args)
    else:
        run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
