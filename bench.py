#!/usr/bin/env python3
"""Throughput of the GB300 Hough-transform track finder on seeded synthetic workloads.

One step = one event through the whole hot path on the GPU: hit staging, stage-1 vote, peak
search, membership and the stage-2 vote.  Default workload: the single high-pileup event
(5,000 helices + 50,000 noise hits, 512 q/pT x 2048 phi0 layer masks, >= 7 layers, 64 x 64
stage 2).  Inputs are resident in HBM before the timed region; L2 is flushed (a 256 MiB write)
before every timed step and each step is bracketed by CUDA events on the launching stream.
A second pass of the same steps with an event after every kernel attributes the step time;
`roofline` is the kernel with the largest share, `kernels` has all of them.

Also reported: `batched` (the batch workload, 256 events of 100-10,000 helices, as one CUDA-graph
replay per step), `served` (Poisson arrivals at 5k/20k/50k events/s through the continuous-
batching server against one launch per event), `e2e` (the public one-call entry point
hough_process from pinned host buffers: host->device copy of the hits, the path, and the
device->host read of the candidate list, timed on the host around each call), `scatter_mode`
(the paper's shared-atomic vote design in place of the gather vote), `count_accumulator` (cells
holding vote counts, the paper's literal A[B[i]] += 1, on the pileup event and the paper's grid),
`d0_axis` (non-prompt tracks on a (d0, q/pT, phi0) grid), `fused_vote_peak` (the vote and the
peak search in one kernel, the accumulator kept in shared memory, against the separate kernels),
`paper_sweep` (the paper's Fig. 2 experiment) and `cpu_baseline` (the FP64 oracle on this
machine's host cores, on a bounded sample; beside it, as context, `fp32_openmp`: the FP32 OpenMP
CPU implementation in the paper's CPU manner on the three single-event workloads).

`--impl reference` times the FP64 CPU oracle (the plain restatement of the method the CUDA path is
checked against) on the host cores, on the same workload and metric.

Launch: `python bench.py [--gpus 1] [--steps K] [--warmup W]`; for N > 1 under
`python -m torch.distributed.run --nproc-per-node N ... bench.py --gpus N`: every rank processes
its own events (events are independent; no collective on the data path) and the timing is the
maximum over ranks.
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

from paper_1310_7556_gb300 import eventgen as eg  # noqa: E402
from paper_1310_7556_gb300 import replicas  # noqa: E402

METRIC = "Hough votes/s and events/s on 1 GB300 (batched vs plain); p50/p99 event latency"
WORKLOAD_TEXT = {
    "pileup_100k": "single high-pileup event: 5000 helices (q=+-1, pT log-uniform 0.5-100 GeV, eta +-2.5, "
                   "z0~N(0,5cm)) + 50000 uniform noise hits on 10 barrel layers r=4..110 cm, B=3.8 T; "
                   "512 q/pT x 2048 phi0 uint16 layer masks, threshold >=7, 64 cot x 64 z0 stage 2",
    "single_50trk": "single event: 50 helices pT 1-50 GeV, no noise; 128 q/pT x 256 phi0, threshold >=8",
    "fine_4m": "fine binning: 20000 helices + 200000 noise hits; 1024 q/pT x 4096 phi0, threshold >=7",
    "paper_2048": "the paper's detector (10 layers evenly spaced to 110 cm, 0.4 mm, transverse plane), "
                  "5000 helices pT 1-100 GeV, no noise; 2048 q/pT x 2048 phi0, threshold >=8",
}
# the pileup event on modules within +-0.5 cm of their layer's radius: every vote per hit
WORKLOAD_TEXT["pileup_100k_jittered"] = WORKLOAD_TEXT["pileup_100k"].replace(
    "+ 50000 uniform noise hits", "+ 50000 uniform noise hits, every hit at its layer radius + U(-0.5, 0.5) cm")
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="pileup_100k", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-events", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--only", choices=["all", "plain", "batched", "served", "paper_sweep", "counts", "d0", "fused"],
                    default="all",
                    help="run one part only (for profiling); the default runs everything")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the batch with the default kernel configuration instead of the tuned one")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="offered-load duration per served point")
    ap.add_argument("--serve-loads", default=",".join(str(int(x)) for x in eg.SERVED_OFFERED_LOADS),
                    help="offered loads (events/s), comma-separated")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
            self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def _oracle_event(job):
    """One event of a workload through the oracle (a process-pool task): (votes, seconds)."""
    import oracle
    name, index = job
    w = eg.WORKLOADS[name]
    ev = w.event(index)
    t0 = time.perf_counter()
    res = oracle.run(w.geometry, w.binning, ev)
    return int(res["votes_by_layer"].sum()), time.perf_counter() - t0


def cpu_baseline(workload, n_single: int = 4):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the workload: one
    thread on n_single events, then one event per core in spawned processes (the oracle is
    single-threaded; an event is its unit of parallel work)."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    t0 = time.perf_counter()
    votes = sum(_oracle_event((workload, i))[0] for i in range(n_single))
    dt1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_event, [(workload, 0)] * cores)   # start-up and first-touch outside the timing
        t0 = time.perf_counter()
        res = pool.map(_oracle_event, [(workload, 100 + i) for i in range(cores)])
        dtn = time.perf_counter() - t0
    return {"value": cores / dtn, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} full {workload} events (seeds 100..{99 + cores}), one per core in spawned "
                      f"processes, whole path (vote, peaks, membership, stage 2), FP64",
            "votes_per_s": sum(v for v, _ in res) / dtn, "seconds": dtn,
            "single_thread": {"value": n_single / dt1, "unit": "events/s", "cores": 1,
                              "sample": f"{n_single} full {workload} events (seeds 0..{n_single - 1})",
                              "votes_per_s": votes / dt1, "seconds": dt1}}


def fp32_baseline(workload, seconds: float = 3.0):
    """The FP32 OpenMP CPU implementation (baseline/hough_cpu.c, the paper's CPU recipe of Sec. 6.2:
    threads over the hits with thread-private accumulators merged at the end, over the rows of the
    peak search and over the candidates) on every host core: events of the workload, one after
    another, for about `seconds` after one untimed event."""
    import baseline
    w = eg.WORKLOADS[workload]
    b = baseline.make_binning(w.geometry, w.binning)
    cores = os.cpu_count() or 1
    baseline.run_event(b, w.event(0), threads=cores)
    n, t0 = 0, time.perf_counter()
    while True:
        baseline.run_event(b, w.event(200 + n), threads=cores)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or n >= 200:
            break
    return {"value": n / dt, "unit": "events/s", "cores": cores, "kind": "fp32_openmp",
            "sample": f"{n} full {workload} events (seeds 200..{199 + n}), one after another, each on all "
                      f"{cores} threads, whole path (vote, peaks, membership, stage 2), FP32", "seconds": dt}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, one event (or a bounded sample) per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = eg.WORKLOADS[args.workload]
    ev = w.event(0)
    # keep the whole run within a few minutes: above 60 steps a step is a prefix sample of the hits
    frac = min(1.0, 60.0 / max(1, args.steps + args.warmup))
    sample = ev if frac >= 1.0 else ev.subset(np.arange(int(ev.n_hits * frac)))
    for _ in range(args.warmup):
        oracle.run(w.geometry, w.binning, sample)
    t0 = time.perf_counter()
    votes = 0
    for _ in range(args.steps):
        votes += int(oracle.run(w.geometry, w.binning, sample)["votes_by_layer"].sum())
    dt = time.perf_counter() - t0
    value = args.steps * frac / dt
    desc = ("one full event per step" if frac >= 1.0 else
            f"per step the first {sample.n_hits} of {ev.n_hits} hits; events/s scaled by that fraction "
            "(the vote is linear in the hits)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "hits": int(ev.n_hits)},
            "votes_per_s": votes / frac / dt if frac > 0 else None,
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Env:
    """Torch, the optional process group, the library binding and the device of this rank."""

    def __init__(self):
        import torch
        import torch.distributed as dist

        from paper_1310_7556_gb300 import binding
        self.torch, self.dist, self.binding = torch, dist, binding
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        if self.world > 1:
            dist.init_process_group(replicas.backend_for(True), device_id=torch.device("cuda", self.local))
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        binding.load()
        self.stream = torch.cuda.current_stream(self.dev)
        self.flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=self.dev)

    def max_over_ranks(self, x: float) -> float:
        return replicas.max_over_ranks(self.dist if self.world > 1 else None, x, device=self.dev)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()
        self.torch.cuda.synchronize()


def measure_plain(env, args, ctx, tens, n):
    """One event per step through hough_vote, hough_peaks, hough_stage2 on device-resident hits.

    The headline steps run with the library's per-kernel events off; a second pass of the same
    steps with them on attributes the step time to kernels."""
    torch, binding, stream = env.torch, env.binding, env.stream

    def step():
        ctx.vote(*tens, n_hits=n, where=binding.DEVICE, stream=stream)
        ctx.peaks(stream=stream)
        ctx.stage2(stream=stream)

    def timed_steps(steps, attribute):
        """K steps, each after an L2 flush, bracketed by CUDA events on the launching stream."""
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        lib_t = []
        for k in range(steps):
            env.flush.zero_()
            e0[k].record(stream)
            step()
            e1[k].record(stream)
            if attribute:
                lib_t.append(ctx.timing())
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in zip(e0, e1)], lib_t

    ctx.enable_timing(False)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    st = ctx.stats()
    env.barrier()
    launches0 = binding.kernel_launches()
    step_ms, _ = timed_steps(args.steps, False)
    launches = binding.kernel_launches() - launches0
    total_ms = env.max_over_ranks(sum(step_ms))
    env.barrier()
    # attribution pass: the same steps with an event after every kernel
    ctx.enable_timing(True)
    step()
    attr_ms, lib_t = timed_steps(min(args.steps, 50), True)
    kernel_ms = {k: statistics.mean(t[k] for t in lib_t) for k in lib_t[0]}
    out = {"events_per_s": replicas.job_rate(args.steps, env.world, total_ms * 1e-3), "ms_per_step": total_ms / args.steps,
           "stage_ms": kernel_ms, "attributed_ms_per_step": statistics.mean(attr_ms),
           "votes": int(st.votes), "general_votes": int(st.general_votes), "candidates": int(st.n_candidates),
           "members": int(st.n_members), "stage2_votes": int(st.stage2_votes), "launches": int(launches)}
    # the same steps with the shared-atomic scatter vote (the paper's GPU design) for comparison, in
    # a few tile shapes (q/pT rows x phi0 columns x threads), the fastest reported
    tiling0 = ctx.get_tiling()
    best = None
    for rows, cols, threads in ((32, 256, 1024), (27, 256, 1024), (32, 128, 1024), (32, 256, 512)):
        if binding.grid_rows(ctx.binning) < rows or ctx.binning.n_phi % cols:
            continue
        ctx.set_tiling(vote_mode=binding.VOTE_SCATTER, tile_qpt=rows, tile_phi=cols, threads=threads)
        for _ in range(3):
            step()
        sc_ms, sc_t = timed_steps(min(args.steps, 20), True)
        r = {"events_per_s": len(sc_ms) / (sum(sc_ms) * 1e-3), "ms_per_step": statistics.mean(sc_ms),
             "vote_ms": statistics.mean(t["vote_ms"] for t in sc_t),
             "peaks_ms": statistics.mean(t["peaks_ms"] for t in sc_t),
             "tile": {"tile_qpt": rows, "tile_phi": cols, "threads": threads}}
        if best is None or r["vote_ms"] < best["vote_ms"]:
            best = r
    ctx.set_tiling(**tiling0)
    ctx.enable_timing(False)
    out["scatter"] = best
    return out


# Kernels of one plain step: (name, timing key, source file that defines it).  Their algorithmic
# work per launch is kernel_work's model below.
PLAIN_KERNELS = [
    ("clear_kernel", "clear_ms", "stage_kernels.cu"),
    ("stage_count_kernel", "count_ms", "stage_kernels.cu"),
    ("table_scan_kernel", "table_ms", "stage_kernels.cu"),
    ("hit_sort_kernel", "sort_ms", "stage_kernels.cu"),
    ("gather_kernel", "gather_ms", "vote_kernel.cu"),
    ("scatter_kernel (vote of per-vote layers)", "scatter_ms", "vote_kernel.cu"),
    ("peaks_kernel", "band_peaks_ms", "vote_kernel.cu"),
    ("compact_kernel", "compact_ms", "vote_kernel.cu"),
    ("confirm_kernel", "stage2_ms", "confirm_kernels.cu"),
]
SMEM_PEAK_HOW = ("hough_microbench_smem_or: 32-bit shared-memory atomicOr, the 32 lanes of a warp on 32 different "
                 "banks, persistent grid of 152-multiple CTAs, measured in this run (not in MEASURED_PEAKS.json)")


def kernel_work(name, w, n_hits, st):
    """Algorithmic work of one launch on one event (or a batch): (bytes, votes or None).

    bytes: what the step must read and write, each once -- hits 13 B (r, phi, z, layer), 2 B per
    accumulator cell written by the vote and read by the peak search, 8 B per band candidate and
    40 B per listed candidate, and for the confirmation 64 B per candidate record (read and
    written), 28 B per (candidate, layer) of table entries, stage-2 terms and bucket offsets, and
    8 B per member (its azimuth fraction and z).  votes: stage-1 votes for the vote kernels, stage-2
    votes for the confirmation: the unit of the shared-atomic ceiling."""
    b = w.binning
    L = w.geometry.n_layers
    cells = st["cells"]
    nkeys = L * b.n_phi * st["events"]
    cands = st["candidates"]
    general = st["general_votes"] / max(1, st["votes"])
    model = {
        "clear_kernel": (4 * nkeys + 8 * 16 * (b.n_phi + 16) * st["events"] + 304, None),
        "stage_count_kernel": (37 * n_hits, None),            # r, phi, z, layer in; key, rank, 16-B record out
        "table_scan_kernel": (8 * nkeys + 32 * 16, None),     # bucket counts in, offsets out; layer records
        "hit_sort_kernel": (72 * n_hits, None),     # key, rank, record, r, phi, z, offset in; 2 x 16 B + f + z out
        "gather_kernel": (13 * n_hits + 2 * cells, st["votes"] - st["general_votes"]),
        "scatter_kernel (vote of per-vote layers)": (13 * n_hits * general, st["general_votes"]),
        "peaks_kernel": (2 * cells + 8 * cands, None),
        "compact_kernel": (40 * cands, None),
        "confirm_kernel": (64 * cands + 28 * L * cands + 8 * st["members"], st["stage2_votes"]),
    }
    staging = ("clear_kernel", "stage_count_kernel", "table_scan_kernel", "hit_sort_kernel")
    model["staging (clear, count, table and scan, hit sort)"] = (sum(model[k][0] for k in staging), None)
    model["compact_kernel + cand_scan_kernel"] = (model["compact_kernel"][0] + 8 * st["events"], None)
    return model[name]


# Steps of a batch as hough_batch_profile times them.
BATCH_STEPS = [
    ("staging (clear, count, table and scan, hit sort)", "stage_ms", "stage_kernels.cu"),
    ("gather_kernel", "gather_ms", "vote_kernel.cu"),
    ("scatter_kernel (vote of per-vote layers)", "scatter_ms", "vote_kernel.cu"),
    ("peaks_kernel", "band_peaks_ms", "vote_kernel.cu"),
    ("compact_kernel + cand_scan_kernel", "compact_ms", "vote_kernel.cu"),
    ("confirm_kernel", "stage2_ms", "confirm_kernels.cu"),
]


def _sources_digest(src):
    import hashlib
    h = hashlib.sha256()
    for f in (src, "hough_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1310_7556_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload, src):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, or None when
    there is none or the kernel's sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic.txt")
    try:
        with open(path) as f:
            lines = [ln.rstrip("\n").split("\t") for ln in f if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    digest = _sources_digest(src)
    for parts in lines:
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[3] == digest:
            return float(parts[2])
    return None


def roofline_entry(ms, nbytes, votes, smem_peak, hbm_peak, peaks_kind):
    """One kernel's rooflines: algorithmic bytes against the measured HBM copy rate and, for the
    vote kernels, votes against the measured shared-atomic ceiling (the blueprint's two ceilings)."""
    sec = ms * 1e-3
    e = {"ms": ms, "hbm": {"algorithmic_bytes": nbytes, "achieved_gbs": nbytes / sec / 1e9 if sec > 0 else None,
                           "peak_gbs": hbm_peak, "frac": nbytes / sec / 1e9 / hbm_peak if sec > 0 else None,
                           "peak_kind": f"{peaks_kind}: MEASURED_PEAKS.json hbm_gbs (STREAM-style copy)"}}
    if votes is not None:
        e["smem_atomic"] = {"votes": votes, "achieved_votes_per_s": votes / sec if sec > 0 else None,
                            "peak_votes_per_s": smem_peak, "frac": votes / sec / smem_peak if sec > 0 else None,
                            "peak_kind": SMEM_PEAK_HOW}
    e["bound"] = "smem_atomic" if votes is not None else "hbm"
    return e


def kernel_table(w, n_hits, st, smem_peak, hbm_peak, peaks_kind, steps=PLAIN_KERNELS):
    """Per-kernel rooflines of one step from its attributed device times (st: counts and stage_ms)."""
    total = sum(st["stage_ms"][k] for _, k, _ in steps)
    table = {}
    for name, key, src in steps:
        ms = st["stage_ms"][key]
        if ms == 0.0 and name in ("clear_kernel", "compact_kernel"):
            continue   # not launched for this event (the state was clean; stage 2 read the band lists)
        nbytes, votes = kernel_work(name, w, n_hits, st)
        e = roofline_entry(ms, float(nbytes), None if votes is None else float(votes), smem_peak, hbm_peak, peaks_kind)
        e["share"] = ms / total if total else None
        e["source"] = src
        table[name] = e
    return table


def headline_roofline(table, dominant, traffic):
    """The bench line's roofline object for the dominant kernel: its votes against the shared-atomic
    ceiling when it votes, else its algorithmic bytes against HBM, with the other beside it."""
    d = table[dominant]
    if d["bound"] == "smem_atomic":
        sa = d["smem_atomic"]
        r = {"kernel": dominant, "bound": "smem_atomic", "achieved": sa["achieved_votes_per_s"],
             "peak": sa["peak_votes_per_s"], "unit": "votes/s", "frac": sa["frac"], "peak_kind": sa["peak_kind"]}
    else:
        h = d["hbm"]
        r = {"kernel": dominant, "bound": "hbm", "achieved": h["achieved_gbs"], "peak": h["peak_gbs"],
             "unit": "GB/s", "frac": h["frac"], "peak_kind": h["peak_kind"]}
    r.update({"traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write)",
              "hbm": d["hbm"], "ms": d["ms"], "share_of_step": d.get("share")})
    return r


def measure_batched(env, args):
    """The batch workload (events of 100-10,000 tracks plus 0.5-2x noise hits): one replayed CUDA graph per
    step over all events of the batch."""
    torch, binding, stream = env.torch, env.binding, env.stream
    wb = eg.WORKLOADS["batch_256"]
    bev = [wb.event(i) for i in replicas.event_indices(env.rank, env.world, args.batch_events)]
    bhs = np.zeros(len(bev) + 1, dtype=np.int64)
    bhs[1:] = np.cumsum([e.n_hits for e in bev])
    bdev = [torch.from_numpy(np.concatenate([getattr(e, k) for e in bev])).to(env.dev) for k in ("r", "phi", "z", "layer")]
    batch = binding.HoughBatch(wb.geometry, wb.binning, max_events=len(bev), max_hits=int(bhs[-1]),
                               max_candidates=1 << 18, max_members=1 << 21, device=env.local)
    for _ in range(3):
        batch.run(*bdev, bhs, where=binding.DEVICE, stream=stream)
    torch.cuda.synchronize()
    # the kernel configuration from the autotuner, chosen on these events before anything is timed
    tune = batch.autotune(*bdev, bhs, where=binding.DEVICE, reps=2) if args.autotune else None
    for _ in range(3):
        batch.run(*bdev, bhs, where=binding.DEVICE, stream=stream)
    torch.cuda.synchronize()
    bstats = [batch.stats(e) for e in range(len(bev))]
    b0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.batch_steps)]
    b1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.batch_steps)]
    env.barrier()
    launch0 = binding.kernel_launches()
    for k in range(args.batch_steps):
        env.flush.zero_()
        b0[k].record(stream)
        batch.run(*bdev, bhs, where=binding.DEVICE, stream=stream)
        b1[k].record(stream)
    torch.cuda.synchronize()
    launches = binding.kernel_launches() - launch0
    total = env.max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(b0, b1)))
    votes = sum(int(st.votes) for st in bstats)
    # attribution: the same run kernel by kernel (hough_batch_profile), an event after each step
    prof = []
    for _ in range(3):
        env.flush.zero_()
        prof.append(batch.profile(*bdev, bhs, where=binding.DEVICE, stream=stream))
    bst = {"events": len(bev), "cells": len(bev) * binding.grid_rows(wb.binning) * wb.binning.n_phi, "votes": votes,
           "general_votes": sum(int(st.general_votes) for st in bstats),
           "candidates": sum(int(st.n_candidates) for st in bstats),
           "members": sum(int(st.n_members) for st in bstats),
           "stage2_votes": sum(int(st.stage2_votes) for st in bstats),
           "stage_ms": {k: statistics.mean(p[k] for p in prof) for k in prof[0]}}
    out = {"events_per_s": replicas.job_rate(len(bev) * args.batch_steps, env.world, total * 1e-3),
           "votes_per_s": replicas.job_rate(votes * args.batch_steps, env.world, total * 1e-3),
           "ms_per_batch": total / args.batch_steps, "events_per_batch": len(bev), "hits_per_batch": int(bhs[-1]),
           "votes_per_batch": votes, "candidates_per_batch": sum(int(st.n_candidates) for st in bstats),
           "members_per_batch": sum(int(st.n_members) for st in bstats),
           "stage2_votes_per_batch": sum(int(st.stage2_votes) for st in bstats),
           "steps": args.batch_steps, "gpu_launches": int(launches),
           "mode": "one CUDA-graph replay per batch; kernels span all events",
           "stage_ms_profiled": bst["stage_ms"]}
    if getattr(args, "smem_peak", None):
        table = kernel_table(wb, int(bhs[-1]), bst, args.smem_peak, args.hbm_peak, args.peaks_kind, BATCH_STEPS)
        dominant = max(table, key=lambda k: table[k]["ms"])
        out["kernels"] = table
        out["roofline"] = headline_roofline(table, dominant,
                                            measured_traffic(dominant, "batch_256", table[dominant]["source"]))
    if tune is not None:
        out["autotune"] = {"tiling": {f: getattr(tune.tiling, f) for f in binding.TILING_FIELDS},
                           "ms_per_batch": tune.ms, "default_ms_per_batch": tune.default_ms,
                           "configurations_timed": tune.tried}
    batch.close()
    return out


def _percentiles(lat_ms):
    if not lat_ms:
        return {"p50_ms": None, "p99_ms": None, "p999_ms": None, "max_ms": None}
    a = np.sort(np.asarray(lat_ms))
    q = lambda p: float(a[min(len(a) - 1, int(math.ceil(p * len(a))) - 1)])
    return {"p50_ms": q(0.50), "p99_ms": q(0.99), "p999_ms": q(0.999), "max_ms": float(a[-1])}


def drive_server(env, srv, pool, rate, seconds, seed, threads=4):
    """Offer a Poisson stream of `rate` events/s for `seconds` to a server through the library's
    trigger emulator (native submitter threads, each submitting at the scheduled arrival; latency
    counts from that time, so a late submission is charged to the server; one native thread polls
    every admitted event)."""
    binding = env.binding
    n = max(1, int(rate * seconds))
    arrivals = eg.poisson_arrivals(rate, n, seed)
    start = binding.serve_clock_ns() + 50_000_000
    at = (start + arrivals * 1e9).astype(np.int64)
    st0 = srv.stats()
    res = srv.replay(pool, at, threads)
    st1 = srv.stats()
    admitted = res["ticket"] != 0
    done = res["done_ns"][admitted]
    lat_ms = ((done - res["arrival_ns"][admitted]) * 1e-6).tolist()
    late_us = (res["submit_ns"][admitted] - res["arrival_ns"][admitted]) * 1e-3
    queue_ms = (res["launch_ns"][admitted] - res["arrival_ns"][admitted]) * 1e-6
    service_ms = (done - res["launch_ns"][admitted]) * 1e-6
    statuses = {}
    for v in res["status"][admitted].tolist():
        statuses[str(v)] = statuses.get(str(v), 0) + 1
    span_s = (int(done.max()) - start) * 1e-9 if done.size else float("nan")
    n_adm = int(admitted.sum())
    return {"offered_ev_s": rate, "seconds": seconds, "offered": n, "admitted": n_adm,
            "dropped": n - n_adm, "dropped_frac": (n - n_adm) / n,
            "completed_ev_s": n_adm / span_s if done.size else 0.0,
            **_percentiles(lat_ms),
            "mean_batch_events": float(res["batch_events"][admitted].mean()) if n_adm else 0.0,
            "max_in_flight": int(st1.max_in_flight), "launches": int(st1.launches - st0.launches),
            "submit_late_p99_us": float(np.percentile(late_us, 99)) if n_adm else None,
            "queue_ms_p50_p99": [float(np.percentile(queue_ms, 50)), float(np.percentile(queue_ms, 99))] if n_adm else None,
            "service_ms_p50_p99": [float(np.percentile(service_ms, 50)), float(np.percentile(service_ms, 99))] if n_adm else None,
            "submitter_threads": threads, "statuses": statuses}


def measure_served(env, args):
    """Trigger-style serving of batch-workload events arriving as Poisson streams: continuous
    batching (events admitted while others run join the next launch; launches overlap on the
    device), in a latency and a throughput setting, against one launch per event through the same
    admission and lanes."""
    binding = env.binding
    wb = eg.WORKLOADS["batch_256"]
    pool_events = [wb.event(i) for i in replicas.event_indices(env.rank, env.world, 64, base=1000)]
    pool = [tuple(np.ascontiguousarray(getattr(e, k)) for k in ("r", "phi", "z", "layer")) for e in pool_events]
    max_event_hits = max(e.n_hits for e in pool_events)
    loads = [float(x) for x in args.serve_loads.split(",") if x]
    # batches of up to 16 events, three launches in flight: the latency setting; batches of up to
    # 64 events, two in flight: the throughput setting (larger launches, a longer tail)
    modes = {"continuous_batching": dict(lanes=4, max_in_flight=3, max_batch_events=16,
                                         max_batch_hits=max(16 * 60_000, max_event_hits)),
             "continuous_batching_large": dict(lanes=3, max_in_flight=2, max_batch_events=64,
                                               max_batch_hits=max(64 * 60_000, max_event_hits)),
             "one_launch_per_event": dict(lanes=2, max_in_flight=1, max_batch_events=1,
                                          max_batch_hits=max_event_hits)}
    out = {"workload": "Poisson arrivals of batch-workload events (100-10,000 helices + 0.5-2x noise hits each; "
                       "a pool of 64 seeded events reused cyclically)",
           "latency": "result on the host minus scheduled arrival",
           "memory_budget_bytes": 48 << 30}
    launch0 = binding.kernel_launches()
    for name, cfg in modes.items():
        srv = binding.HoughServer(wb.geometry, wb.binning, max_candidates=1 << 17, max_members=1 << 21,
                                  memory_budget=48 << 30, lane_timeout_us=30_000_000, device=env.local, **cfg)
        # warm: one of each pool event through the server
        for e in pool[:8]:
            t = None
            while t is None:
                t = srv.submit(e[0], e[1], e[2], e[3], e[0].shape[0])
            srv.poll(t, timeout_us=60_000_000, candidates=False)
        # and a short saturating burst, so that the result buffers have grown to full batches
        drive_server(env, srv, pool, 50_000.0, 0.5, seed=5)
        res = []
        for k, rate in enumerate(loads):
            res.append(drive_server(env, srv, pool, rate, args.serve_seconds, seed=77 + k))
        st = srv.stats()
        out[name] = {"config": {**cfg, "lanes_in_service": int(st.lanes), "device_bytes": int(st.device_bytes)},
                     "loads": res}
        srv.close()
    out["gpu_launches"] = int(binding.kernel_launches() - launch0)
    return out


def measure_paper_sweep(env, args):
    """The paper's timing experiment (Fig. 2: time per event against the number of tracks on its
    detector and 2048 x 2048 grid) on this GPU: the plain path, one event per step, device-resident
    hits, L2 flushed before every step; and the FP64 oracle single-threaded on the host, at the
    sizes it finishes within a few seconds."""
    import oracle
    torch, binding, stream = env.torch, env.binding, env.stream
    points = []
    oracle.build()
    for nt in eg.PAPER_TRACK_COUNTS:
        w = eg.paper_workload(nt)
        ev = w.event(0)
        tens = [torch.from_numpy(np.ascontiguousarray(a)).to(env.dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]
        with binding.HoughContext(w.geometry, w.binning, max_hits=max(ev.n_hits, 1), max_candidates=1 << 18,
                                  max_members=1 << 22, device=env.local) as ctx:
            def step():
                ctx.vote(*tens, n_hits=ev.n_hits, where=binding.DEVICE, stream=stream)
                ctx.peaks(stream=stream)
                ctx.stage2(stream=stream)
            for _ in range(3):
                step()
            torch.cuda.synchronize()
            st = ctx.stats()
            k = 50
            e0 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
            e1 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
            for q in range(k):
                env.flush.zero_()
                e0[q].record(stream)
                step()
                e1[q].record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in zip(e0, e1))
        p = {"tracks": nt, "hits": int(ev.n_hits), "votes": int(st.votes), "candidates": int(st.n_candidates),
             "gpu_ms_per_event": ms, "gpu_events_per_s": 1e3 / ms}
        if nt <= 2000 or nt == eg.PAPER_TRACK_COUNTS[-1]:
            t0 = time.perf_counter()
            oracle.run(w.geometry, w.binning, ev)
            p["oracle_ms_per_event_1_thread"] = (time.perf_counter() - t0) * 1e3
        points.append(p)
    return {"workload": WORKLOAD_TEXT["paper_2048"].replace("5000 helices", "N helices"), "points": points}


def count_workloads():
    """The count accumulator's workloads: (name, workload, what it is)."""
    acc = eg.ACC_COUNTS
    return [
        ("pileup_100k", eg.with_binning(eg.WORKLOADS["pileup_100k"], accumulator=acc, threshold=70),
         WORKLOAD_TEXT["pileup_100k"].replace("uint16 layer masks, threshold >=7",
                                              "uint16 vote counts, threshold >=70 votes (about 48 per cell)")),
        ("paper_2048_500", eg.with_binning(eg.paper_workload(500), accumulator=acc, threshold=8),
         WORKLOAD_TEXT["paper_2048"].replace("5000 helices", "500 helices").replace(
             "threshold >=8", "uint16 vote counts, threshold >=8 votes")),
    ]


def _plain_variant(env, args, w, text, smem_peak=None, hbm_peak=None):
    """One configuration of the plain path, one event per step, device-resident hits, L2 flushed
    before every step; then an attribution pass with an event after every kernel."""
    torch, binding, stream = env.torch, env.binding, env.stream
    ev = w.event(replicas.event_indices(env.rank, env.world, 1)[0])
    tens = [torch.from_numpy(np.ascontiguousarray(a)).to(env.dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]
    tune = None
    if args.autotune:
        # the kernel configuration from the autotuner, timed on a one-event batch of this event
        with binding.HoughBatch(w.geometry, w.binning, max_events=1, max_hits=max(ev.n_hits, 1),
                                max_candidates=1 << 18, max_members=1 << 23, device=env.local) as tb:
            tune = tb.autotune(*tens, np.array([0, ev.n_hits], dtype=np.int64), where=binding.DEVICE, reps=5)
    with binding.HoughContext(w.geometry, w.binning, max_hits=max(ev.n_hits, 1), max_candidates=1 << 18,
                              max_members=1 << 23, device=env.local) as ctx:
        if tune is not None:
            ctx.set_tiling(**{f: getattr(tune.tiling, f) for f in binding.TILING_FIELDS})

        def step():
            ctx.vote(*tens, n_hits=ev.n_hits, where=binding.DEVICE, stream=stream)
            ctx.peaks(stream=stream)
            ctx.stage2(stream=stream)

        def timed(k, attribute):
            e0 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
            e1 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
            lib_t = []
            for q in range(k):
                env.flush.zero_()
                e0[q].record(stream)
                step()
                e1[q].record(stream)
                if attribute:
                    lib_t.append(ctx.timing())
            torch.cuda.synchronize()
            return [a.elapsed_time(b) for a, b in zip(e0, e1)], lib_t

        ctx.enable_timing(False)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        st = ctx.stats()
        env.barrier()
        step_ms, _ = timed(args.steps, False)
        total = env.max_over_ranks(sum(step_ms))
        ctx.enable_timing(True)
        step()
        _, lib_t = timed(min(args.steps, 30), True)
        ctx.enable_timing(False)
        t = {k: statistics.mean(x[k] for x in lib_t) for k in lib_t[0]}
        tiling = ctx.get_tiling()
    cells = binding.grid_rows(w.binning) * w.binning.n_phi
    vote_ms = t["vote_ms"]
    p = {"workload": text, "hits": int(ev.n_hits), "cells": cells, "votes": int(st.votes),
         "general_votes": int(st.general_votes), "refined_votes": int(st.refined_votes),
         "candidates": int(st.n_candidates), "members": int(st.n_members),
         "events_per_s": replicas.job_rate(args.steps, env.world, total * 1e-3), "ms_per_event": total / args.steps,
         "stage_ms": t["stage_ms"], "vote_ms": vote_ms, "gather_ms": t["gather_ms"], "scatter_ms": t["scatter_ms"],
         "peaks_ms": t["peaks_ms"], "stage2_ms": t["stage2_ms"],
         "votes_per_s_in_vote": st.votes / (vote_ms * 1e-3) if vote_ms > 0 else None,
         "vote_mode": "gather" if tiling["vote_mode"] == binding.VOTE_GATHER else "scatter",
         "tiling": tiling, "tiling_from": "autotuner (one-event batch)" if tune is not None else "default"}
    if smem_peak and vote_ms > 0:
        p["vote_vs_smem_atomic_peak"] = p["votes_per_s_in_vote"] / smem_peak
    if hbm_peak and vote_ms > 0:
        gbs = (13 * ev.n_hits + 2 * cells) / (vote_ms * 1e-3) / 1e9
        p["vote_hbm"] = {"achieved_gbs": gbs, "frac": gbs / hbm_peak, "algorithmic": "13 B per hit in, 2 B per cell out"}
    return p


def measure_counts(env, args, smem_peak=None, hbm_peak=None):
    """The count accumulator (A[B[i]] += 1 of Sec. 8: a cell holds its number of votes, saturating
    at 65535; the shared-memory scatter kernel votes, the peak search reads counts)."""
    return {name: _plain_variant(env, args, w, text, smem_peak, hbm_peak) for name, w, text in count_workloads()}


def measure_d0(env, args, smem_peak=None, hbm_peak=None):
    """Non-prompt tracks: the (d0, q/pT, phi0) grid of the displaced workload, with layer masks and
    with counts."""
    w = eg.WORKLOADS["displaced_d0"]
    text = ("displaced tracks: 200 helices pT 2-100 GeV with d0 ~ U(-2, 2) cm (eta +-2.5, z0~N(0,5cm)) + 1000 "
            "noise hits on 10 barrel layers r=4..110 cm, B=3.8 T; 16 d0 (+-2 cm) x 256 q/pT (+-1) x 2048 phi0 "
            "uint16 {}, threshold >=8, 3x3x3 peaks, 64 cot x 64 z0 stage 2")
    wc = eg.with_binning(w, accumulator=eg.ACC_COUNTS)
    return {"layers": _plain_variant(env, args, w, text.format("layer masks"), smem_peak, hbm_peak),
            "counts": _plain_variant(env, args, wc, text.format("vote counts"), smem_peak, hbm_peak)}


def measure_fused(env, args):
    """The fused vote and peak search (vote_mode HOUGH_VOTE_FUSED: the accumulator stays in shared
    memory) against the default separate kernels: the plain step on the pileup event for a sweep
    of band heights and block sizes, and a 64-event batch of the batch workload; L2 flushed before
    every timed step.  The fused candidates are checked equal to the default ones."""
    torch, binding, stream = env.torch, env.binding, env.stream
    w = eg.WORKLOADS["pileup_100k"]
    ev = w.event(replicas.event_indices(env.rank, env.world, 1)[0])
    tens = [torch.from_numpy(np.ascontiguousarray(a)).to(env.dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]

    def timed(step, k):
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        for q in range(k):
            env.flush.zero_()
            e0[q].record(stream)
            step()
            e1[q].record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in zip(e0, e1))

    plain = {}
    with binding.HoughContext(w.geometry, w.binning, max_hits=ev.n_hits, max_candidates=1 << 18,
                              max_members=1 << 23, device=env.local) as ctx:
        def step():
            ctx.vote(*tens, n_hits=ev.n_hits, where=binding.DEVICE, stream=stream)
            ctx.peaks(stream=stream)
            ctx.stage2(stream=stream)
        base = ctx.get_tiling()
        k = max(10, min(args.steps, 50))
        plain["default"] = timed(step, k)
        ref = ctx.candidates(stream=stream).copy()
        same = True
        for r in (2, 4, 8):
            for th in (512, 1024):
                ctx.set_tiling(**{**base, "vote_mode": binding.VOTE_FUSED, "band_rows": r, "gather_threads": th})
                plain[f"fused band_rows={r} threads={th}"] = timed(step, k)
                same = same and np.array_equal(ctx.candidates(stream=stream), ref)
    best = min((v, name) for name, v in plain.items() if name != "default")
    wb = eg.WORKLOADS["batch_256"]
    events = [wb.event(i) for i in replicas.event_indices(env.rank, env.world, 64)]
    hs = np.zeros(len(events) + 1, dtype=np.int64)
    hs[1:] = np.cumsum([e.n_hits for e in events])
    cat = lambda name, dt: torch.from_numpy(np.concatenate([getattr(e, name) for e in events]).astype(dt)).to(env.dev)
    bt = [cat("r", np.float32), cat("phi", np.float32), cat("z", np.float32), cat("layer", np.uint8)]
    batch = {}
    with binding.HoughBatch(wb.geometry, wb.binning, max_events=len(events), max_hits=int(hs[-1]),
                            device=env.local) as b:
        def bstep():
            b.run(*bt, hs, where=binding.DEVICE, stream=stream)
        for name, kw in (("default", {}), ("fused band_rows=8 threads=512", dict(vote_mode=binding.VOTE_FUSED, band_rows=8,
                                                                                 gather_threads=512)),
                         ("fused band_rows=16 threads=512", dict(vote_mode=binding.VOTE_FUSED, band_rows=16,
                                                                 gather_threads=512))):
            b.set_tiling(**kw)
            batch[name] = timed(bstep, 5)
    return {"workload": WORKLOAD_TEXT["pileup_100k"] + "; and 64 events of the batch workload",
            "plain_ms_per_event": plain, "best_fused": best[1], "best_fused_vs_default": best[0] / plain["default"],
            "fused_candidates_equal_default": bool(same),
            "batch64_ms_per_batch": batch,
            "note": "vote_mode HOUGH_VOTE_FUSED computes each band of full rows with its two halo rows in shared "
                    "memory and searches it there; the accumulator is not written"}


def measure_e2e(env, args, ctx, ev):
    """hough_process from pinned host buffers: hits to the device, the path, candidates back."""
    torch, stream = env.torch, env.stream
    n = ev.n_hits
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (ev.r, ev.phi, ev.z, ev.layer)]
    out = np.zeros(1 << 18, dtype=env.binding.CANDIDATE_DTYPE)
    for _ in range(3):
        ctx.process(*pinned, n_hits=n, out=out, stream=stream)
    env.barrier()
    e2e_s = []
    got = None
    for _ in range(args.steps):
        env.flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = ctx.process(*pinned, n_hits=n, out=out, stream=stream)
        e2e_s.append(time.perf_counter() - t0)
    total = env.max_over_ranks(sum(e2e_s))
    return {"value": replicas.job_rate(args.steps, env.world, total), "unit": "events/s",
            "h2d_bytes_per_step": n * (4 + 4 + 4 + 1),
            "d2h_bytes_per_step": len(got) * 32 + 160}


def served_headline(served):
    """Completed events/s and latency percentiles of each served setting at each offered load."""
    if not served:
        return None
    out = {}
    for mode in ("continuous_batching", "continuous_batching_large"):
        if mode in served:
            out[mode] = {str(int(p["offered_ev_s"])): {"completed_ev_s": p["completed_ev_s"], "p50_ms": p["p50_ms"],
                                                        "p99_ms": p["p99_ms"], "dropped_frac": p["dropped_frac"]}
                         for p in served[mode]["loads"]}
    return out


def measure_per_vote_path(env, args, smem_peak, hbm_peak):
    """The pileup event on a detector whose modules sit within +-0.5 cm of their layer's radius: no
    layer's hits share one radius, so every stage-1 vote is evaluated per hit in the shared-atomic
    scatter kernel (FP32 arcsine, FP64 near a bin edge) -- the path the gather cannot take."""
    w = eg.WORKLOADS["pileup_100k_jittered"]
    p = _plain_variant(env, args, w, WORKLOAD_TEXT["pileup_100k_jittered"], smem_peak, hbm_peak)
    p["note"] = "all votes cast by scatter_kernel (vote of per-vote layers); vote_vs_smem_atomic_peak is its rate"
    return p


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    env = Env()
    binding = env.binding
    if args.only == "batched":
        peaks, args.peaks_kind = measured_peaks()
        args.hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
        args.smem_peak = binding.smem_or_throughput(env.local, 0, 30.0)
    if args.only in ("batched", "served", "paper_sweep", "counts", "d0", "fused"):
        out = {"batched": measure_batched, "served": measure_served, "paper_sweep": measure_paper_sweep,
               "counts": measure_counts, "d0": measure_d0, "fused": measure_fused}[args.only](env, args)
        if env.rank == 0:
            print(json.dumps({"metric": METRIC, "part": args.only, **out}), flush=True)
        return

    w = eg.WORKLOADS[args.workload]
    ev = w.event(replicas.event_indices(env.rank, env.world, 1)[0])     # each rank its own event
    n = ev.n_hits
    tens = [env.torch.from_numpy(np.ascontiguousarray(a)).to(env.dev) for a in (ev.r, ev.phi, ev.z, ev.layer)]
    ctx = binding.HoughContext(w.geometry, w.binning, max_hits=n, max_candidates=1 << 18,
                               max_members=1 << 23, device=env.local)
    plain_tune = None
    if args.autotune:
        # the kernel configuration from the autotuner, timed on a one-event batch of this event
        hs1 = np.array([0, n], dtype=np.int64)
        with binding.HoughBatch(w.geometry, w.binning, max_events=1, max_hits=n, max_candidates=1 << 18,
                                max_members=1 << 23, device=env.local) as tb:
            plain_tune = tb.autotune(*tens, hs1, where=binding.DEVICE, reps=10)
        ctx.set_tiling(**{f: getattr(plain_tune.tiling, f) for f in binding.TILING_FIELDS})
    # measured shared-atomic ceiling (conflict-free 32-lane atomicOr), before anything is timed
    smem_peak = binding.smem_or_throughput(env.local, 0, 30.0)
    smem_peak_rand = binding.smem_or_throughput(env.local, 1, 30.0)
    peaks, peaks_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    args.smem_peak, args.hbm_peak, args.peaks_kind = smem_peak, hbm_peak, peaks_kind
    with ClockSampler(env.local) as clock_sampler:
        plain = measure_plain(env, args, ctx, tens, n)
        per_vote = measure_per_vote_path(env, args, smem_peak, hbm_peak)
        if args.only == "plain":
            batched = e2e = served = paper = counts = d0 = fused = None
        else:
            batched = measure_batched(env, args)
            e2e = measure_e2e(env, args, ctx, ev)
            served = measure_served(env, args)
            paper = measure_paper_sweep(env, args) if env.rank == 0 else None
            counts = measure_counts(env, args, smem_peak, hbm_peak)
            d0 = measure_d0(env, args, smem_peak, hbm_peak)
            fused = measure_fused(env, args)
    clocks = clock_sampler.summary()
    st = dict(plain, events=1, cells=binding.grid_rows(w.binning) * w.binning.n_phi)
    kernels = kernel_table(w, n, st, smem_peak, hbm_peak, peaks_kind)
    dominant = max(kernels, key=lambda k: kernels[k]["ms"])
    src = dict((name, s) for name, _, s in PLAIN_KERNELS)[dominant]
    traffic = measured_traffic(dominant, args.workload, src)
    votes = plain["votes"]
    scatter = plain.pop("scatter")
    scatter["votes_per_s_in_vote_kernel"] = votes / (scatter["vote_ms"] * 1e-3)
    scatter["smem_atomic_frac"] = scatter["votes_per_s_in_vote_kernel"] / smem_peak
    line = {
        "metric": METRIC,
        "value": plain["events_per_s"],
        "unit": "events/s",
        "n_gpus": env.world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": plain["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        # the other headline figures first, so that a truncated copy of this line keeps them
        "batched_events_per_s": batched["events_per_s"] if batched else None,
        "batched_votes_per_s": batched["votes_per_s"] if batched else None,
        "batched_ms_per_256_events": batched["ms_per_batch"] if batched else None,
        "served": served_headline(served),
        "config": {"workload": WORKLOAD_TEXT[args.workload], "hits": n, "votes_per_event": votes,
                   "candidates_per_event": plain["candidates"], "members_per_event": plain["members"],
                   "stage2_votes_per_event": plain["stage2_votes"],
                   "mode": "plain: one event per step, hough_vote + hough_peaks + hough_stage2 (7 kernel launches)",
                   "l2": "flushed before every timed step (256 MiB write)", "tiling": ctx.get_tiling(),
                   "tiling_from": "autotuner (one-event batch, 10 replays per configuration)" if plain_tune else "default"},
        "votes_per_s": votes * plain["events_per_s"],
        "roofline": headline_roofline(kernels, dominant, traffic),
        "batched_roofline": batched.get("roofline") if batched else None,
        "kernels": kernels,
        "smem_atomic_peak": {"conflict_free": smem_peak, "random_words": smem_peak_rand,
                             "unit": "lane atomicOr/s", "how": SMEM_PEAK_HOW},
        "scatter_mode": scatter,
        "per_vote_path": per_vote,
        "batched": batched,
        "served_detail": served,
        "paper_sweep": paper,
        "count_accumulator": counts,
        "d0_axis": d0,
        "fused_vote_peak": fused,
        "e2e": e2e,
        "gpu_launches": plain["launches"],
        "clocks": clocks,
    }
    if env.rank == 0 and env.world == 1 and not args.no_cpu_baseline and args.only == "all":
        line["cpu_baseline"] = cpu_baseline(args.workload)
        # context: the FP32 multi-core CPU implementation on the three single-event workloads
        line["cpu_baseline"]["fp32_openmp"] = {k: fp32_baseline(k) for k in ("single_50trk", "pileup_100k", "fine_4m")}
    ctx.close()
    if env.rank == 0:
        print(json.dumps(line), flush=True)
    if env.world > 1:
        env.dist.destroy_process_group()


if __name__ == "__main__":
    main()
