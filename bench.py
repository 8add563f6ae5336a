#!/usr/bin/env python
"""Throughput of the cell-list neighbor query + RDF on 4,194,304 points (one GB300).

Workload (one step): N = 4,194,304 uniform points in a cubic box at density 0.85 (seeded,
synthetic, shaped like the paper's random-point benchmarks); build the cell list; ball
query r_max = 2.5 producing the full sorted NeighborList (~2.33e8 pairs); fused RDF of
500 bins on [0, 5] (~1.87e9 ordered pairs, never stored).  value = neighbor pairs
handled per second = (NeighborList pairs + RDF pairs) / step time.  Under torchrun the
ranks split that one frame by ranges of query cells (each holds every point, writes the
rows of its own queries and histograms its own pairs; the counts and the histogram are
summed over NCCL), so the value is the frame's pairs over the slowest rank's time.

Timing: W untimed warm-up steps; K timed steps, each bracketed by CUDA events on the
launching stream; L2 is flushed (a 512 MB write) before every step outside the events;
barrier + synchronize around the timed region; max over ranks.  Per-kernel device times
come from libfgb's own CUDA events over the same region.  `e2e` repeats the step through
the public API from pinned host memory (H2D of the points and D2H of the RDF counts and
pair total inside the events).  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload on all host cores.
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

import workloads as W  # noqa: E402

L2_BYTES = 129 * 2 ** 20
ORACLE_SAMPLE = 1 << 20  # queries of the workload the CPU oracle times (cpu_baseline)
ORACLE_BLOCKS = 4        # ... in this many equal blocks spread over the query indices
REFERENCE_SAMPLE = 1 << 18  # queries per step of --impl reference


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def frame_seed(rank: int) -> int:
    """The c3 frame's seed.  Under torchrun every rank holds the same frame and walks its
    own range of the query cells (strong scaling over one frame)."""
    return 3


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over all ranks (the step time every rank waits for)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_rank: int, world: int, step_ms: float) -> float:
    """Whole-job throughput when every rank processes its own units: all ranks' units over
    the slowest rank's time."""
    return units_per_rank * world / (step_ms * 1e-3)


def strong_value(units: int, step_ms: float) -> float:
    """Whole-job throughput when the ranks split one frame: its units over the slowest
    rank's time."""
    return units / (step_ms * 1e-3)


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per launch of the top kernels from one ncu capture of the
# c3 workload at 2,097,152 points (profiles/k_*_c3_2M.md), with the sha256 prefix of the
# captured build's sources (the kernel's file, then the tile header it inlines).
# Traffic grows in proportion to N at fixed density, so it is scaled to the bench's N;
# once a source changes the figure is stale and is reported as null.
_NL = ("paper_1906_06317_gb300/csrc/nlist.cu", "paper_1906_06317_gb300/csrc/fgb_tile.cuh")
_RDF = ("paper_1906_06317_gb300/csrc/rdf.cu", "paper_1906_06317_gb300/csrc/fgb_tile.cuh")
MEASURED_TRAFFIC = {
    "k_nl_write": (_NL, "6793fdff82cf7609", 576.290560e6 + 1544.660e6, 2097152),
    "k_nl_count": (_NL, "6793fdff82cf7609", 42.768896e6 + 0.072e6, 2097152),
    "k_rdf_tile": (_RDF, "3eddbba7d02e9b5d", 34.218496e6 + 0.005888e6, 2097152),
}


# Shared-atomic wavefronts of the fused RDF as a share of the shared-memory data pipe's
# peak (ncu l1tex__data_pipe_lsu_wavefronts_mem_shared_op_atom, the same capture).
MEASURED_SHARED_ATOMICS = {
    "k_rdf_tile": (_RDF, "3eddbba7d02e9b5d", 0.1174),
}


def _sources_sha(paths) -> str:
    import hashlib
    d = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            d.update(f.read())
    return d.hexdigest()


def measured_shared_atomics(kernel: str):
    """Measured fraction of the shared pipe's peak taken by atomics, or None when stale."""
    if kernel not in MEASURED_SHARED_ATOMICS:
        return None
    paths, sha, frac = MEASURED_SHARED_ATOMICS[kernel]
    try:
        cur = _sources_sha(paths)
    except OSError:
        return None
    return frac if cur.startswith(sha) else None


def measured_traffic(kernel: str, n: int):
    """Scaled DRAM bytes per launch, or None when unmeasured or the source has changed."""
    if kernel not in MEASURED_TRAFFIC:
        return None
    paths, sha, nbytes, n0 = MEASURED_TRAFFIC[kernel]
    try:
        cur = _sources_sha(paths)
    except OSError:
        return None
    return nbytes * n / n0 if cur.startswith(sha) else None


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), architecture and cores."""
    import platform
    fields = {}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            fields.setdefault(k.strip(), v.strip())
    except (OSError, subprocess.SubprocessError):
        pass
    name = fields.get("Model name") or fields.get("Vendor ID") or ""
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return f"{name or 'unknown'} ({platform.machine()}, {os.cpu_count()} logical cores)"


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------------ oracle arm


def oracle_blocks(n: int, sample: int, blocks: int):
    """`blocks` equal ranges of query indices, `sample` queries in all, spread evenly over
    [0, n) (the points are i.i.d., so each range is a uniform spatial sample)."""
    blocks = max(1, min(blocks, sample))
    size = sample // blocks
    return [(k * n // blocks, k * n // blocks + size) for k in range(blocks)]


def oracle_rate(w, sample: int, threads: int, blocks: int = 1):
    """Pairs per second of the CPU oracle on `sample` queries (in `blocks` spread ranges),
    with the O(N) cell-list builds charged in proportion (sample / N)."""
    import oracle
    p = w.params
    n = len(w.points)
    t0 = time.perf_counter()
    c_nl = oracle.Cells(w.box, w.points, p["r_max"])
    c_rdf = oracle.Cells(w.box, w.points, p["rdf_r_max"])
    t_cells = time.perf_counter() - t0
    del c_nl, c_rdf
    rg = oracle_blocks(n, sample, blocks)
    pairs = 0
    t1 = time.perf_counter()
    for q in rg:
        counts, _, _, _ = oracle.ball_query(w.box, w.points, p["r_max"], queries=q, threads=threads)
        h = oracle.rdf_counts(w.box, w.points, p["rdf_bins"], p["rdf_r_max"], queries=q, threads=threads)
        pairs += int(counts.sum()) + int(h.sum())
    t_q = time.perf_counter() - t1
    done = sum(b - a for a, b in rg)
    # each oracle call builds its own cell list over all N points (two per block); charge
    # those builds only in proportion to the fraction of the workload the sample covers
    t = t_q - t_cells * (len(rg) - done / n)
    return pairs / t, pairs, t


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = W.c3()
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_rate(w, REFERENCE_SAMPLE // 8, threads)
    rates, times = [], []
    for _ in range(args.steps):
        r, pairs, t = oracle_rate(w, REFERENCE_SAMPLE, threads)
        rates.append(r)
        times.append(t)
    v = statistics.median(rates)
    sample = (f"queries [0, {REFERENCE_SAMPLE}) of {len(w.points)} per step (ball r=2.5 + RDF 500 bins [0,5]); "
              "cell builds charged pro rata")
    line = {"impl": "reference", "metric": "neighbor pairs/s (cell-list query+RDF) at N=4M", "value": v,
            "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "c3: cubic rho=0.85, N=4194304 uniform, ball r=2.5 NL + RDF 500 bins [0,5]",
                       "oracle_sample": sample},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the kNN / Q6 / batch component timings")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--points", type=int, default=4_194_304,
                    help="points of the uniform workload (smaller cases are for profiling only)")
    ap.add_argument("--only", choices=["pmft", "batch", "q6", "knn", "tree"], default=None,
                    help="time one group of components alone and print them (profiling runs)")
    ap.add_argument("--pmft-points", type=int, default=4_194_304, help="points of the large 2D PMFT frame")
    ap.add_argument("--batch-frames", type=int, default=256, help="--only batch: the first frames of the c5 set")
    args = ap.parse_args()
    rank, world, local = env_rank()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_1906_06317_gb300 as fgb

    torch.cuda.set_device(local)
    if args.only == "pmft":
        dev = torch.device("cuda", local)
        flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
        comp = pmft_components(fgb, torch, dev, torch.cuda.current_stream(), flush, n_big=args.pmft_points)
        print(json.dumps({"components": comp}), flush=True)
        return
    if args.only in ("q6", "knn", "tree"):
        dev = torch.device("cuda", local)
        flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
        comp = component_only(fgb, torch, dev, torch.cuda.current_stream(), flush, args.only, args.points,
                              args.steps, args.warmup)
        print(json.dumps({"components": comp}), flush=True)
        return
    if args.only == "batch":
        dev = torch.device("cuda", local)
        flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
        comp = batch_only(fgb, torch, dev, torch.cuda.current_stream(), flush, args.batch_frames, args.steps,
                          args.warmup)
        print(json.dumps({"components": comp}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    w = W.c3(seed=frame_seed(rank), n=args.points)
    p = w.params
    host = torch.from_numpy(w.points).pin_memory()
    pts = host.to(dev)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    rdf = fgb.RDF(p["rdf_bins"], p["rdf_r_max"])
    stream = torch.cuda.current_stream()

    if world > 1:
        from paper_1906_06317_gb300 import shard

    capacity = {"pairs": 0}

    def step(x):
        nq = fgb.NeighborQuery(w.box, x, r_cell=p["r_max"])
        if world > 1:
            # one frame split across the ranks by ranges of query cells; the counts and
            # the histogram are summed over NCCL
            shard.sharded_rdf(rdf, nq, rank, world, all_reduce=dist.all_reduce)
            return shard.sharded_ball_query(nq, p["r_max"], rank, world, all_reduce=dist.all_reduce)
        rdf.compute(nq, reset=True)
        # the list is queued without a host synchronisation into arrays sized from the
        # previous frame's list (+2 %); its completion checks the status words it copied back
        return nq.query_async(p["r_max"], exclude_ii=True, capacity=capacity["pairs"])

    for _ in range(max(3, args.warmup)):
        nl = step(pts)
        if world == 1:
            capacity["pairs"] = int(nl.n_pairs * 1.02)
    torch.cuda.synchronize()
    nl_pairs = int(nl.global_segments[-1]) if world > 1 else nl.n_pairs
    nl_esc = 0 if world > 1 else nl.escalations
    rdf_pairs = int(rdf.bin_counts.sum())
    rdf_esc = rdf.escalations()
    units = nl_pairs + rdf_pairs
    del nl

    # ---------------- timed region (device-resident inputs)
    fgb.timing_reset()
    fgb.timing_enable(True)
    launches0 = fgb.kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                          if world == 1 else local)
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nl = step(pts)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        if world == 1:
            assert not nl.wait().rewritten      # every timed list fit its arrays as queued
        del nl
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    launches = (fgb.kernel_launches() - launches0) // args.steps
    fgb.timing_enable(False)
    kern = {}
    for name in ("k_bin", "k_radix_hist", "k_radix_scatter", "k_cell_start", "k_ball_count", "k_ball_write",
                 "k_ball_write_global", "k_tile_count", "k_tile_write", "k_nl_count", "k_nl_count_scatter",
                 "k_nl_write", "k_nl_fill_qi", "k_tile_write_listed", "k_tile_write_global_listed",
                 "k_sort_segments", "k_rdf_tile", "k_reduce", "k_top", "k_down", "k_rdf", "k_rdf_escalated",
                 "k_offset_table", "k_origin_tables", "k_band"):
        t, n = fgb.timing_read(name)
        if n:
            kern[name] = {"ms_per_step": t / args.steps, "launches_per_step": n / args.steps}
    step_ms = sum(ms) / len(ms)
    # FP64 decisions inside the FP32 bands, per pair (one step's list and histogram)
    esc = {"nl_fp64_decisions": int(nl_esc), "nl_fraction_of_pairs": nl_esc / max(nl_pairs, 1),
           "rdf_fp64_decisions": int(rdf_esc), "rdf_fraction_of_unordered_pairs": rdf_esc / max(rdf_pairs / 2, 1)}
    step_ms_max = max_over_ranks(step_ms, dist, dev)
    value = strong_value(units, step_ms_max)

    # ---------------- end to end through the public API, host buffers
    e2e_ms = []
    for k in range(max(2, min(args.steps, 5))):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x = host.to(dev, non_blocking=True)
        nl = step(x)
        counts = rdf.bin_counts           # D2H of the step's result (synchronises)
        got = int(counts.sum()) + (int(nl.global_segments[-1]) if world > 1 else nl.n_pairs)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        assert got == units
        del nl, x
    e2e_step = max_over_ranks(statistics.median(e2e_ms), dist, dev)

    # ---------------- roofline of the dominant kernel
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    n = len(w.points)
    dominant = max(kern, key=lambda k: kern[k]["ms_per_step"])
    sm_clock = (clk or {}).get("sm_max_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sms * 128 * sm_clock * 1e6 / 1e12   # FP32 lane-instructions per second, T/s
    rdf_unordered = rdf_pairs / 2
    nl_bytes = (12.0 * nl_pairs + 28.0 * n) / 1e9    # 12 B per stored pair; record, count, offset per query
    cnt_bytes = 20.0 * n / 1e9                        # sorted record read + count write per query
    # write kernel: point index + distance (+ query index unless a fill pass stores it) per
    # pair; sorted record, count and offset per query
    nlw_bytes = ((8.0 if "k_nl_fill_qi" in kern else 12.0) * nl_pairs + 28.0 * n) / 1e9
    qi_bytes = (4.0 * nl_pairs + 8.0 * n) / 1e9      # query index per pair; offset per query
    rdf_ops = 10.0 * rdf_unordered / 1e12             # ~10 FP32 operations per unordered pair inside r_max
    roofs = {
        "k_ball_write": ("hbm", nl_bytes, "GB/s", hbm),
        "k_tile_write": ("hbm", nl_bytes, "GB/s", hbm),
        "k_ball_count": ("hbm", cnt_bytes, "GB/s", hbm),
        "k_tile_count": ("hbm", cnt_bytes, "GB/s", hbm),
        "k_nl_write": ("hbm", nlw_bytes, "GB/s", hbm),
        "k_nl_fill_qi": ("hbm", qi_bytes, "GB/s", hbm),
        "k_nl_count": ("hbm", cnt_bytes, "GB/s", hbm),
        "k_rdf": ("alu", rdf_ops, "TOP/s", alu_peak),
        "k_rdf_tile": ("alu", rdf_ops, "TOP/s", alu_peak),
    }
    bound, work, unit, peak = roofs.get(dominant, ("hbm", 0.0, "GB/s", hbm))
    t_dom = kern[dominant]["ms_per_step"] / kern[dominant]["launches_per_step"] * 1e-3
    achieved = work / t_dom
    roofline = {"kernel": dominant, "bound": bound, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak, "traffic": measured_traffic(dominant, n),
                "traffic_unit": "bytes per launch (ncu dram read+write, scaled from 2,097,152 points)",
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if bound == "hbm"
                else f"derived: {n_sms} SMs x 128 FP32 lanes x {sm_clock:.0f} MHz"}
    others = {}
    for k, (b, wk, u, pk) in roofs.items():
        if k in kern:
            tk = kern[k]["ms_per_step"] / kern[k]["launches_per_step"] * 1e-3
            others[k] = {"bound": b, "achieved": wk / tk, "peak": pk, "unit": u, "frac": wk / tk / pk,
                         "ms": tk * 1e3, "traffic": measured_traffic(k, n)}
            sa = measured_shared_atomics(k)
            if sa is not None:
                others[k]["shared_atomics_frac_of_peak"] = sa

    # ---------------- other parts of the hot path (component timings)
    components = {}
    if not args.no_extras and rank == 0:
        components = extras(fgb, torch, dev, stream, flush)

    # ---------------- CPU oracle baseline (rank 0, N=1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r, pairs, t = oracle_rate(w, ORACLE_SAMPLE, threads, ORACLE_BLOCKS)
        r1, pairs1, t1 = oracle_rate(w, ORACLE_SAMPLE // 128, 1)
        blocks = ", ".join(f"[{a}, {b})" for a, b in oracle_blocks(n, ORACLE_SAMPLE, ORACLE_BLOCKS))
        cpu = {"value": r, "unit": "pairs/s", "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": f"queries {blocks} of {n}: {pairs} pairs in {t:.1f} s (cell builds charged pro rata)",
               "single_thread": {"value": r1, "unit": "pairs/s", "cores": 1,
                                 "sample": f"queries [0, {ORACLE_SAMPLE // 128}) of {n}: {pairs1} pairs in "
                                           f"{t1:.1f} s"}}

    if rank == 0:
        line = {"metric": "neighbor pairs/s (cell-list query+RDF) at N=4M", "value": value, "unit": "pairs/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms_max,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": "c3: cubic rho=0.85, N=4194304 uniform, cell list r=2.5, ball r=2.5 full "
                                       "sorted NeighborList + fused RDF 500 bins [0,5]",
                           "nl_pairs": nl_pairs, "rdf_pairs": rdf_pairs, "points_per_rank": n,
                           "l2": "flushed (512 MB write) before every step", "parallelism": "one frame" if world == 1 else
                           f"one frame over {world} ranks: query-cell slabs, counts and histogram summed (NCCL)"},
                "e2e": {"value": strong_value(units, e2e_step), "unit": "pairs/s",
                        "h2d_bytes_per_step": int(host.numel() * 4), "d2h_bytes_per_step": p["rdf_bins"] * 8},
                "gpu_launches": int(launches), "roofline": roofline, "kernels": kern, "kernel_rooflines": others,
                "escalations": esc,
                "components": components, "clocks": clk, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def timed(fn, stream, flush, reps=5, warm=2):
    import torch
    for _ in range(warm):
        fn()
    out = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def component_only(fgb, torch, dev, stream, flush, which, n_points, steps, warmup):
    """One component alone, `warmup` then `steps` timed runs: the commands behind the
    captures of its kernels.  q6: Q6 forward + backward on the c4 system (2^20 points,
    fixed list r = 1.3); knn: k = 12 on the c3 workload with n_points points (cell list
    built each run); tree: tree build + ball query r = 2.5 on the same points."""
    if which == "q6":
        w4 = W.c4()
        x4 = torch.from_numpy(w4.points).to(dev)
        nq4 = fgb.NeighborQuery(w4.box, x4, r_cell=1.3)
        nl4 = nq4.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
        st = fgb.Steinhardt(6)

        def fn():
            st.compute(nq4, neighbors=nl4)
            st.backward(1.0)
        label = "c4_q6_fwd_bwd_ms"
    else:
        w = W.c3(n=n_points)
        x = torch.from_numpy(w.points).to(dev)
        if which == "knn":
            r12 = (3.0 * 13 / (4.0 * math.pi * 0.85)) ** (1.0 / 3.0)

            def fn():
                nq = fgb.NeighborQuery(w.box, x, r_cell=1.35 * r12)
                return nq.query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()
            label = "c3_knn12_ms"
        else:
            def fn():
                aq = fgb.AABBQuery(w.box, x)
                return aq.query(None, dict(r_max=2.5, exclude_ii=True)).toNeighborList()
            label = "c3_tree_build_query_ms"
    for _ in range(warmup):
        fn()
    return {label: timed(fn, stream, flush, reps=max(steps, 1), warm=0), "points": n_points if which != "q6" else 2 ** 20}


def batch_only(fgb, torch, dev, stream, flush, n_frames, steps, warmup):
    """The c5 frames [0, n_frames) in one batch at fixed settings (cell size r_max, tile
    items of up to 64 cells, 4 query cells per warp), `warmup` then `steps` plain runs
    (no graph, no tuning): the command behind the batch kernels' launch lists and
    captures."""
    frames = W.c5()[:n_frames]
    P = W.C5_PARAMS
    sizes = [len(f.points) for f in frames]
    pts = torch.from_numpy(np.concatenate([f.points for f in frames])).to(dev)
    b = fgb.Batch(sizes, [f.box for f in frames], r_max=P["r_max"], l=P["l"], rdf_bins=P["rdf_bins"],
                  rdf_r_max=P["rdf_r_max"], cell_div=1, block=128, hist_copies=2, tile_cells=64, cells_per_warp=4)
    for _ in range(warmup):
        b.run(pts)
    ms = timed(lambda: b.run(pts), stream, flush, reps=max(steps, 1), warm=0)
    return {"batch_frames": len(frames), "batch_points": int(sum(sizes)), "batch_ms": ms, "routes": b.routes()}


def pmft_components(fgb, torch, dev, stream, flush, n_big=4_194_304):
    """PMFT(x, y) next to the RDF on 2D systems (the comparison of Fig. 6): the paper's
    10 frames x 20,000 points at 12 neighbours per unit disc, PMFT on [-1, 1)^2 with
    100 x 100 bins and the RDF with 100 bins out to the PMFT's reach sqrt(2), each frame
    with its own cell list; then one 4,194,304-point frame at the same density."""
    comp = {}
    prm = W.P6_PARAMS
    xm, ym, bx, by = prm["x_max"], prm["y_max"], prm["bins_x"], prm["bins_y"]
    reach = math.hypot(xm, ym)
    frames = W.p6()
    fx = [(f.box, torch.from_numpy(f.points).to(dev), torch.from_numpy(f.theta).to(dev)) for f in frames]
    pm = fgb.PMFTXY(xm, ym, (bx, by))
    rdf = fgb.RDF(bx, reach)

    def p6_pmft():
        for k, (b, x, t) in enumerate(fx):
            pm.compute(fgb.NeighborQuery(b, x, r_cell=reach), t, reset=(k == 0))

    def p6_rdf():
        for k, (b, x, t) in enumerate(fx):
            rdf.compute(fgb.NeighborQuery(b, x, r_cell=reach), reset=(k == 0))

    t_pm, t_rdf = timed(p6_pmft, stream, flush), timed(p6_rdf, stream, flush)
    comp["p6_fig6_10x20000_pmft_ms"] = t_pm
    comp["p6_fig6_10x20000_rdf_ms"] = t_rdf
    comp["p6_pmft_over_rdf"] = t_pm / t_rdf
    # one large 2D frame: the fused kernels' throughput in bonds within reach per second
    n = n_big
    big = W.p6(seed=61, n=n, n_frames=1)[0]
    xb, tb = torch.from_numpy(big.points).to(dev), torch.from_numpy(big.theta).to(dev)
    nqb = fgb.NeighborQuery(big.box, xb, r_cell=reach)
    bonds = nqb.query(None, dict(r_max=reach, exclude_ii=True)).toNeighborList().n_pairs
    t_big = timed(lambda: pm.compute(nqb, tb, reset=True), stream, flush)
    esc = pm.escalations()
    # per-kernel device time of the fused route (CUDA events around each launch)
    fgb.timing_reset()
    fgb.timing_enable(True)
    for _ in range(3):
        flush.zero_()
        pm.compute(nqb, tb, reset=True)
    torch.cuda.synchronize()
    fgb.timing_enable(False)
    per = {}
    for k in ("k_pmft_trig_sorted", "k_pmft_tile", "k_pmft_escalated"):
        t, c = fgb.timing_read(k)
        per[k] = t / max(c, 1)
    peaks = measured_peaks()
    sm_clock = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sms * 128 * sm_clock * 1e6 / 1e12
    # 32 FP32 operations per unordered pair within reach: displacement 2, r^2 2, and per
    # direction rotation 4, bin index 2, floor 2, fraction 2, margin tests 4
    ops = 32.0 * (bonds / 2) / 1e12
    tile_s = per["k_pmft_tile"] * 1e-3
    roof = {"kernel": "k_pmft_tile", "bound": "alu", "achieved": ops / tile_s, "peak": alu_peak, "unit": "TOP/s",
            "frac": ops / tile_s / alu_peak, "ms": per["k_pmft_tile"],
            "peak_source": f"derived: {n_sms} SMs x 128 FP32 lanes x {sm_clock:.0f} MHz"}
    t_bigr = timed(lambda: rdf.compute(nqb, reset=True), stream, flush)
    nl_holder = {}

    def list_route():
        nl_holder["nl"] = nqb.query(None, dict(r_max=reach * (1 + 1e-6), exclude_ii=True)).toNeighborList()
        pm.compute(nqb, tb, neighbors=nl_holder["nl"], reset=True)

    t_list = timed(list_route, stream, flush, reps=3, warm=1)
    t_list_only = timed(lambda: pm.compute(nqb, tb, neighbors=nl_holder["nl"], reset=True), stream, flush, reps=3,
                        warm=1)
    comp["pmft_2d_%dk" % (n // 1024)] = {"points": n, "pmft_ms": t_big, "rdf_ms": t_bigr, "pmft_list_route_ms": t_list, "pmft_from_stored_list_ms": t_list_only, "bonds": bonds,
                          "pmft_bonds_per_s": bonds / t_big * 1e3, "escalated": esc,
                                               "kernel_ms": per, "roofline": roof}
    return comp


def extras(fgb, torch, dev, stream, flush):
    comp = {}
    # kNN k=12 on the same 4M-point workload; cells about 1.35x the mean 12th-neighbor
    # distance so one 27-cell stencil covers almost every query
    w = W.c3()
    x = torch.from_numpy(w.points).to(dev)
    r12 = (3.0 * 13 / (4.0 * math.pi * 0.85)) ** (1.0 / 3.0)

    def knn():
        nq = fgb.NeighborQuery(w.box, x, r_cell=1.35 * r12)
        return nq.query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList()

    comp["c3_knn12_ms"] = timed(knn, stream, flush)

    # the same r = 2.5 NeighborList from the tree NeighborQuery (build + query) next to
    # the cell list (build + query)
    def tree_query():
        aq = fgb.AABBQuery(w.box, x)
        return aq.query(None, dict(r_max=2.5, exclude_ii=True)).toNeighborList()

    def cell_query():
        nq = fgb.NeighborQuery(w.box, x, r_cell=2.5)
        return nq.query(None, dict(r_max=2.5, exclude_ii=True)).toNeighborList()

    comp["c3_tree_build_query_ms"] = timed(tree_query, stream, flush, reps=3, warm=1)
    aq3 = fgb.AABBQuery(w.box, x)
    comp["c3_tree_knn12_ms"] = timed(lambda: aq3.query(None, dict(num_neighbors=12, exclude_ii=True)).toNeighborList(),
                                     stream, flush, reps=3, warm=1)
    del aq3
    comp["c3_cell_build_query_ms"] = timed(cell_query, stream, flush, reps=3, warm=1)
    # clustered points (2,000 Gaussian blobs of 1,000, sigma 0.5, overall density 0.1):
    # the same r = 1 list from the tree and from the cell list, checked equal
    wb = W.blobs()
    xb = torch.from_numpy(wb.points).to(dev)
    lists = {}

    def blob_tree():
        lists["tree"] = fgb.AABBQuery(wb.box, xb).query(None, dict(r_max=1.0, exclude_ii=True)).toNeighborList()

    def blob_cells():
        lists["cells"] = fgb.NeighborQuery(wb.box, xb, r_cell=1.0).query(None, dict(r_max=1.0, exclude_ii=True)
                                                                         ).toNeighborList()

    comp["blobs_tree_build_query_ms"] = timed(blob_tree, stream, flush, reps=3, warm=1)
    comp["blobs_cell_build_query_ms"] = timed(blob_cells, stream, flush, reps=3, warm=1)
    assert torch.equal(lists["tree"].point_indices, lists["cells"].point_indices)
    comp["blobs_pairs"] = lists["cells"].n_pairs
    del lists
    # Q6 forward + backward, N = 2^20, fixed neighbor list r = 1.3
    w4 = W.c4()
    x4 = torch.from_numpy(w4.points).to(dev)
    nq4 = fgb.NeighborQuery(w4.box, x4, r_cell=1.3)
    nl4 = nq4.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()
    st = fgb.Steinhardt(6)

    def fwd():
        st.compute(nq4, neighbors=nl4)

    def fwdbwd():
        st.compute(nq4, neighbors=nl4)
        st.backward(1.0)

    comp["c4_q6_fwd_ms"] = timed(fwd, stream, flush)
    comp["c4_q6_fwd_bwd_ms"] = timed(fwdbwd, stream, flush)
    # c1: 4,096 points, L = 16: cell list + ball query r = 4 + RDF 100 bins (latency-bound)
    w1 = W.c1()
    x1 = torch.from_numpy(w1.points).to(dev)
    rdf1 = fgb.RDF(100, 4.0)

    def c1_step():
        nq = fgb.NeighborQuery(w1.box, x1, r_cell=4.0)
        nl = nq.query(None, dict(r_max=4.0, exclude_ii=True)).toNeighborList()
        rdf1.compute(nq, reset=True)
        return nl

    comp["c1_query_rdf_us"] = 1e3 * timed(c1_step, stream, flush)
    # c2: 500,000-point FCC crystal in a triclinic box: ball query r = 1.3, q4 and q6 from
    # the list, RDF 200 bins on [0, 5) (its own cell list at r_max / 2)
    w2 = W.c2()
    x2 = torch.from_numpy(w2.points).to(dev)
    holder = {}

    def c2_query():
        nq = fgb.NeighborQuery(w2.box, x2, r_cell=1.3)
        holder["nq"], holder["nl"] = nq, nq.query(None, dict(r_max=1.3, exclude_ii=True)).toNeighborList()

    comp["c2_ball_query_ms"] = timed(c2_query, stream, flush)
    st4, st6 = fgb.Steinhardt(4), fgb.Steinhardt(6)

    def c2_ql():
        st4.compute(holder["nq"], neighbors=holder["nl"])
        st6.compute(holder["nq"], neighbors=holder["nl"])

    comp["c2_q4_q6_ms"] = timed(c2_ql, stream, flush)
    # Steinhardt variants on the same list: normalised W_6, q6 followed by its neighbor
    # average, and LocalDescriptors with l_max = 6 (49 harmonics of 8 B per bond: an HBM
    # roofline of output bytes + the 8 B index pair read per bond)
    st6.compute(holder["nq"], neighbors=holder["nl"])
    comp["c2_w6_ms"] = timed(lambda: st6.wl(), stream, flush)

    def c2_avg():
        st6.compute(holder["nq"], neighbors=holder["nl"])
        st6.average(holder["nl"])

    comp["c2_q6_plus_average_ms"] = timed(c2_avg, stream, flush)
    ld = fgb.LocalDescriptors(6)
    t_ld = timed(lambda: ld.compute(holder["nq"], holder["nl"]), stream, flush)
    ld_bytes = holder["nl"].n_pairs * (49 * 8 + 8)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    comp["c2_descriptors_l6"] = {"ms": t_ld, "bytes": ld_bytes, "achieved_gbs": ld_bytes / t_ld / 1e6,
                                 "frac_of_measured_hbm": ld_bytes / t_ld / 1e6 / peak}
    ld.sph = None
    # clusters of the whole list, and the solid-liquid parameter (l = 6, 0.7, 7 bonds)
    comp["c2_cluster_ms"] = timed(lambda: fgb.Cluster().compute(holder["nq"], holder["nl"]), stream, flush)
    sl = fgb.SolidLiquid(6, 0.7, 7)
    comp["c2_solid_liquid_ms"] = timed(lambda: sl.compute(holder["nq"], holder["nl"]), stream, flush)
    comp["c2_largest_solid_cluster"] = sl.largest_cluster_size
    rdf2 = fgb.RDF(200, 5.0)

    def c2_rdf():
        rdf2.compute(fgb.NeighborQuery(w2.box, x2, r_cell=2.5), reset=True)

    comp["c2_rdf_ms"] = timed(c2_rdf, stream, flush)
    rdf_l = fgb.RDF(130, 1.3)
    comp["c2_rdf_from_list_ms"] = timed(lambda: rdf_l.compute(holder["nq"], neighbors=holder["nl"], reset=True),
                                        stream, flush)
    comp["c2_nl_pairs"] = holder["nl"].n_pairs
    comp.update(pmft_components(fgb, torch, dev, stream, flush))
    holder.clear()
    # batched frames
    if hasattr(fgb.lib(), "fgb_batch_run"):
        try:
            comp.update(batch_extras(fgb, torch, dev, stream, flush))
        except Exception as e:  # report, do not hide
            comp["c5_error"] = repr(e)
    return comp


def batch_extras(fgb, torch, dev, stream, flush):
    frames = W.c5()
    P = W.C5_PARAMS
    sizes = [len(f.points) for f in frames]
    pts = torch.from_numpy(np.concatenate([f.points for f in frames])).to(dev)
    b = fgb.Batch(sizes, [f.box for f in frames], r_max=P["r_max"], l=P["l"], rdf_bins=P["rdf_bins"],
                  rdf_r_max=P["rdf_r_max"])
    tuned = b.tune(pts)
    t_graph = timed(lambda: b.run(pts, graph=True), stream, flush)
    routes = b.routes()
    # the same frames with every frame on the per-point kernel (its tuned settings)
    bp = fgb.Batch(sizes, [f.box for f in frames], r_max=P["r_max"], l=P["l"], rdf_bins=P["rdf_bins"],
                   rdf_r_max=P["rdf_r_max"], cell_div=1, block=256, hist_copies=1, tile_cells=-1)
    t_point = timed(lambda: bp.run(pts, graph=True), stream, flush)
    del bp
    xs = [torch.from_numpy(f.points).to(dev) for f in frames]
    rdf = fgb.RDF(P["rdf_bins"], P["rdf_r_max"])
    st = fgb.Steinhardt(P["l"])

    def loop():
        for f, xf in zip(frames, xs):
            nq = fgb.NeighborQuery(f.box, xf, r_cell=P["r_max"])
            rdf.compute(nq, reset=True)
            st.compute(nq, neighbors=dict(r_max=P["r_max"], exclude_ii=True))

    t_loop = timed(loop, stream, flush, reps=3, warm=1)
    return {"c5_frames": len(frames), "c5_points": int(sum(sizes)), "c5_batched_graph_ms": t_graph,
            "c5_frames_per_s_batched": len(frames) / (t_graph * 1e-3), "c5_per_frame_loop_ms": t_loop,
            "c5_frames_per_s_per_frame_loop": len(frames) / (t_loop * 1e-3), "c5_tuned": tuned,
            "c5_routes": routes, "c5_per_point_route_graph_ms": t_point}


if __name__ == "__main__":
    main()
