#!/usr/bin/env python3
"""Benchmark of the Hash Chain (HC) searching phase on GB300.

Workload (one "step"): the plain-HC sweep -- four 256 MiB texts drawn i.i.d.
uniform over sigma in {2, 4, 20, 95} symbols, and for each sigma the pattern
lengths m in {2, 4, ..., 1024}; P patterns per (sigma, m) cell (default 100),
each copied from its text at a seeded offset; (q, alpha) as the paper sets
them for that text type and m.  Every pattern is searched over its whole text
and all occurrence positions are produced, in text order.

Metric: text GB/s searched (bytes of text / device time, 1e9), device-timed
with CUDA events on the launching stream, texts resident in HBM; the texts
(256 MiB) are larger than the 129 MB L2, so no flush is needed.  Also
reported: GB/s per cell, the roofline fraction of the search kernel against
the measured HBM bandwidth, an end-to-end figure through the synchronous
C-ABI call with host buffers (host->device text copies and device->host
position reads inside the timed region), the CPU oracle's throughput on the
host cores, and SM clocks sampled during the timed region.

``--impl reference`` times the CPU oracle (the plain C HC of the paper's
Fig. 4/5) instead, on a bounded sample of the same workload.

``--workload skewed`` runs the same measurement on the skewed config: one
1 GiB text from an order-2 Markov source over 60 symbols (Zipf(1.1)
unigrams), m in {4, 8, ..., 1024}, P patterns per m copied from the text.
``--workload batched`` and ``--workload served`` are described at their
functions.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun, one process per GPU, each searching the full sweep (weak scaling,
no collective on the data path).
"""
from __future__ import annotations

import argparse
import gc
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

import hc_inputs as hi  # noqa: E402

GB = 1e9
SERVED_RATES_DEFAULT = (1000, 10000, 50000)
METRIC = "text GB/s searched (device-timed), plain HC sweep"
SKEW_METRIC = "text GB/s searched (device-timed), skewed Markov text"
SKEW_KEY = 60        # the skewed text's alphabet size, its key among the texts
UNIT = "GB/s"


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--patterns", type=int, default=100, help="patterns per (sigma, m) cell")
    ap.add_argument("--n", type=int, default=1 << 28, help="text length per sigma")
    ap.add_argument("--cells", default="",
                    help="comma-separated sigma:m cells to run instead of the whole sweep "
                         "(a small case for profiling, e.g. 4:4); the line is then not the headline")
    ap.add_argument("--params", choices=["tuned", "paper"], default="tuned",
                    help="(q, alpha) and launch options per cell: measured by the autotuner on this "
                         "GPU (default), or the paper's Tables 1-3")
    ap.add_argument("--tuner-table", default="",
                    help="load the autotuner's table from this file if it exists, else calibrate "
                         "and save it there (so that two runs use the same parameters); default: "
                         "the table measured on a GB300 for the workload (profiles/), when the "
                         "device is a GB300, else a fresh calibration")
    ap.add_argument("--retune", action="store_true",
                    help="calibrate the autotuner afresh instead of loading the stored GB300 table")
    ap.add_argument("--pos64", action="store_true",
                    help="positions as uint64 instead of uint32 (the sweep's texts are < 2^32 bytes)")
    ap.add_argument("--eager", action="store_true",
                    help="enqueue every search from Python in the timed steps instead of replaying "
                         "one CUDA graph per step")
    ap.add_argument("--clock-ms", type=int, default=200,
                    help="nvidia-smi sampling interval during the timed region (0: no sampling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="sweep only: skip the skewed, batched and served sub-objects")
    ap.add_argument("--extra-patterns", type=int, default=20,
                    help="patterns per m of the skewed sub-object")
    ap.add_argument("--extra-served-seconds", type=float, default=1.0,
                    help="seconds per offered load of the served sub-object")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", choices=["sweep", "skewed", "batched", "served"], default="sweep",
                    help="sweep: the plain-HC sweep (default); skewed: the 1 GiB order-2 Markov "
                         "text; batched: 4096 queries in one graph-captured batch vs. one plain "
                         "launch per query; served: Poisson request streams into the server vs. "
                         "a plain per-request server")
    ap.add_argument("--skew-n", type=int, default=1 << 30, help="skewed text length")
    ap.add_argument("--served-rates", type=int, nargs="+", default=list(SERVED_RATES_DEFAULT))
    ap.add_argument("--served-seconds", type=float, default=2.0)
    ap.add_argument("--served-reps", type=int, default=3,
                    help="repetitions of each offered load per server (order alternating; latencies pooled)")
    ap.add_argument("--served-backlog", type=int, default=50000,
                    help="requests submitted at once for the saturation measurement")
    ap.add_argument("--batch-queries", type=int, default=4096)
    ap.add_argument("--tune-text-bytes", type=int, default=64 << 20,
                    help="calibration text per alphabet size (batched workload)")
    return ap.parse_args()


def metric_for(args):
    return SKEW_METRIC if getattr(args, "workload", "sweep") == "skewed" else METRIC


def skew_sigma_eff(y: np.ndarray) -> float:
    """Effective alphabet size of a text, 1 / sum of squared symbol
    frequencies (the alphabet size of a uniform text with the same chance
    that two random positions hold the same symbol), from its first 64 MiB."""
    c = np.bincount(y[:1 << 26], minlength=256).astype(np.float64)
    p = c / c.sum()
    return float(1.0 / np.sum(p * p))


def workload_inputs(args, patterns: int):
    """Texts (host arrays keyed by an alphabet size), the (key, m) cells, and
    per cell the patterns, of the sweep or the skewed workload."""
    if getattr(args, "workload", "sweep") == "skewed":
        texts = {SKEW_KEY: hi.skew_text(args.skew_n)}
        grid = [(SKEW_KEY, m) for m in hi.SKEW_MS]
    else:
        grid = [(s, m) for s in hi.SWEEP_SIGMAS for m in hi.SWEEP_MS]
        texts = None
    if args.cells:
        grid = [tuple(int(v) for v in c.split(":")) for c in args.cells.split(",")]
    if texts is None:
        texts = {s: hi.sweep_text(s, args.n) for s in sorted({s for s, _ in grid})}
    pats = {(s, m): hi.sweep_patterns(texts[s], s, m, patterns) for s, m in grid}
    return texts, grid, pats


def workload_config(args):
    if getattr(args, "workload", "sweep") == "skewed":
        return {
            "workload": "plain HC, skewed text",
            "text_bytes": args.skew_n,
            "text": "order-2 Markov source over 60 symbols (bytes 65..124), Zipf(1.1) unigrams, "
                    "seeded transition rows; patterns copied from the text",
            "cells": args.cells or "all",
            "ms": list(hi.SKEW_MS),
            "patterns_per_cell": args.patterns,
            "q_alpha": ("autotuned on uniform calibration texts over the text's effective alphabet "
                        "size (1 / sum of squared symbol frequencies); paper_params gives the "
                        "paper's English column (nearest alphabet size)"
                        if getattr(args, "params", "paper") == "tuned" else
                        "paper's English column (Tables 1-3), the nearest alphabet size"),
            "l2": f"inputs larger than L2 ({args.skew_n >> 20} MiB text vs 129 MB L2); no flush",
            "launch": ("eager enqueue of every search" if getattr(args, "eager", False)
                       else "one CUDA graph per step (all its searches), replayed"),
            "positions": "uint64" if getattr(args, "pos64", False) else "uint32 (texts < 2^32 bytes)",
        }
    return {
        "workload": "plain HC sweep",
        "text_bytes_per_sigma": args.n,
        "sigmas": list(hi.SWEEP_SIGMAS),
        "cells": args.cells or "all",
        "ms": list(hi.SWEEP_MS),
        "patterns_per_cell": args.patterns,
        "text": "i.i.d. uniform uint8, seeds 100+sigma; patterns copied from the text",
        "q_alpha": ("autotuned per (sigma, m) on this GPU (calibration texts of the same kind, not the "
                    "sweep's); paper_params gives the sweep on Tables 1-3"
                    if getattr(args, "params", "paper") == "tuned" else
                    "paper's choice per text type and m (Tables 1-3), q clamped to m"),
        "l2": "inputs larger than L2 (256 MiB texts vs 129 MB L2); no flush",
        "launch": ("eager enqueue of every search" if getattr(args, "eager", False)
                   else "one CUDA graph per step (all its searches), replayed"),
        "positions": "uint64" if getattr(args, "pos64", False) else "uint32 (texts < 2^32 bytes)",
    }


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 200, enabled: bool = True):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.enabled = enabled
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        if not self.enabled:
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.enabled:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (--clock-ms 0)"]}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
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
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def scan_family(m: int, q: int, mode: int = 0) -> str:
    """The scan kernel a search runs: the given mode, else the library's
    automatic choice."""
    if mode:
        return {1: "scan_staged", 2: "scan_direct", 3: "scan_dense"}[mode]
    if m == q:
        return "scan_dense"
    if m - q + 1 >= 200 or m > 16384:
        return "scan_direct"
    return "scan_staged"


TUNER_TABLES = {"sweep": "profiles/tuner_sweep_gb300.txt", "skewed": "profiles/tuner_skewed_gb300.txt",
                "batched": "profiles/tuner_batched_gb300.txt"}


def stored_tuner_table(workload: str, device_name: str, retune: bool):
    """The autotuner's table measured on a GB300 for this workload (the
    parameters the committed profiles and traffic records were taken with),
    used when the device is a GB300; None to calibrate afresh."""
    if retune or "GB300" not in device_name:
        return None
    rel = TUNER_TABLES.get(workload)
    return os.path.join(ROOT, rel) if rel else None


def dense_single_pass(opts, m: int) -> bool:
    """Whether the library runs a dense (m = q) search as its single-pass
    kernel: the same rule as its planner (chunks of 256 * L window starts,
    L even, tiles of at most 64 steps of 512 windows, staging buffers and
    two tiles' step masks within the 227 KB of shared memory per block)."""
    if opts is None or getattr(opts, "single_pass", 0) != 1:
        return False
    lane = opts.lane_bytes if opts is not None and opts.lane_bytes else 16
    stages = opts.stages if opts is not None and opts.stages else 2
    ls = max(2, (lane + 1) & ~1)
    spc = ls // 2
    want = opts.tile_steps if opts is not None and getattr(opts, "tile_steps", 0) else 16
    tc = max(1, -(-want // spc))
    if spc * tc > 64:
        return False
    stage = ((16 + 256 * ls + m - 1 + 15) & ~15) + 32
    return 8 * stages * stage + 8 * 2 * spc * tc * 64 + 1024 <= 227 * 1024


KERNEL_SOURCES = ("paper_2310_15711_gb300/csrc/hc_kernels.cuh", "paper_2310_15711_gb300/csrc/hc_search.cu",
                  "paper_2310_15711_gb300/csrc/hc_device.cuh", "paper_2310_15711_gb300/csrc/hc_dense.cu")


def recorded_traffic(family: str, workload: str = "sweep"):
    """DRAM bytes per launch of a kernel family from the committed ncu record
    (profiles/traffic.json; the sweep's records at the top level, another
    workload's under its name, since a launch's bytes depend on its text):
    None unless the workload has a record for the family taken on the
    current kernel sources.  Returns (bytes per launch, record)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(f.read())
    ent = rec.get(family) if workload == "sweep" else rec.get(workload, {}).get(family)
    if not ent or rec.get("source_sha") != h.hexdigest()[:16]:
        return None, None
    return ent.get("dram_bytes_per_launch"), ent


def recorded_cell_traffic(cell: str, q: int, alpha: int, lane_bytes: int, mode: int,
                          workload: str = "sweep"):
    """DRAM bytes of one search of a direct-scan cell (whose reads skip most
    of the text, so that its bytes are not the text's size) from the
    committed ncu record (profiles/traffic.json, "direct_cells"), when it was
    taken on the current kernel sources with the same q, alpha and launch
    options; else None."""
    _, rec = recorded_traffic("scan_direct", workload)
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if rec is None and not os.path.exists(path):
        return None
    with open(path) as f:
        allrec = json.load(f)
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(f.read())
    if allrec.get("source_sha") != h.hexdigest()[:16]:
        return None
    cells = allrec.get("direct_cells", {}) if workload == "sweep" else allrec.get(workload, {}).get("direct_cells", {})
    ent = cells.get(cell)
    if not ent or (ent.get("q"), ent.get("alpha"), ent.get("lane_bytes"), ent.get("mode")) != (q, alpha, lane_bytes, mode):
        return None
    return ent.get("dram_bytes_per_launch")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
def cpu_baseline(texts, cells, seconds: float, threads: int):
    """The oracle's HC (plain C, unmodified) on the host cores: a bounded
    sample of the sweep -- a prefix of each text, a few patterns per cell --
    until about `seconds` of wall time; returns text GB/s."""
    import oracle
    oracle.build()
    prefix = 1 << 24
    full = max(t.size for t in texts.values())
    total_bytes, total_t, searched = 0, 0.0, 0
    k = 0
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < seconds:
        for (sigma, m), pats in cells.items():
            y = texts[sigma][:prefix]
            x = pats[k % len(pats)]
            q, alpha = hi.paper_q_alpha(sigma, m)
            t0 = time.perf_counter()
            oracle.hc_search_threaded(x, y, q, alpha, threads)
            total_t += time.perf_counter() - t0
            total_bytes += y.size
            searched += 1
        k += 1
    return {"value": total_bytes / total_t / GB, "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": f"{searched} searches: {len(cells)} cells x {k} pattern(s) each, "
                      f"first {prefix >> 20} MiB of each {full >> 20} MiB text, "
                      f"{threads} threads over pieces overlapping by m-1"}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as the reference arm."""
    if rank != 0:
        return
    texts, _, cells = workload_inputs(args, max(1, min(args.patterns, 4)))
    threads = os.cpu_count() or 1
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(texts, cells, 0.5, threads)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(texts, cells, per_step, threads))
    wall = time.perf_counter() - t0
    v = float(np.mean([c["value"] for c in vals]))
    ref_config = dict(workload_config(args))
    ref_config["q_alpha"] = "the paper's choice per text type and m (Tables 1-3), q clamped to m"
    line = {
        "impl": "reference", "metric": metric_for(args), "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": ref_config,
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": vals[-1]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2310_15711_gb300 as hc

    dist = None
    if world > 1:
        import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    hc.build()
    hc.lib()

    # ---- parameters: measured per (sigma, m) on this GPU by the autotuner
    # (single-search path, its own calibration texts), unless --params paper
    texts_np, grid, patterns = workload_inputs(args, args.patterns)
    sigmas = sorted({s for s, _ in grid})
    # the alphabet size the tuner's table is read at: a uniform text's own,
    # the skewed text's effective one
    tune_sigma = {s: (max(2, int(round(skew_sigma_eff(texts_np[s])))) if args.workload == "skewed" else s)
                  for s in sigmas}
    tune_s = None
    tuner = None
    tuner_source = None
    if args.params == "tuned":
        tuner = hc.HCTuner()
        t0 = time.perf_counter()
        table = args.tuner_table or stored_tuner_table(args.workload, torch.cuda.get_device_name(dev),
                                                       args.retune)
        if table and os.path.exists(table):
            tuner.load(table)
            tuner_source = table
        else:
            tuner.calibrate(sorted(set(tune_sigma.values())), sorted({m for _, m in grid}),
                            text_bytes=args.n, seed=21, path=hc.HC_TUNE_SINGLE)
            torch.cuda.synchronize(dev)
            if args.tuner_table:
                tuner.save(args.tuner_table)
            tuner_source = "calibrated in this run"
        tune_s = time.perf_counter() - t0

    # positions as uint32 (the texts are far below 2^32 bytes) unless --pos64
    pos32 = 0 if args.pos64 else 1
    pos_bytes = 8 if args.pos64 else 4

    # ---- inputs
    texts = {s: torch.from_numpy(t).to(dev) for s, t in texts_np.items()}

    def make_cells(kind):
        out = {}
        for s, m in grid:
            pats = patterns[(s, m)]
            if kind == "tuned":
                e = tuner.lookup(tune_sigma[s], m)
                q, alpha = e["q"], e["alpha"]
                opts = hc.SearchOpts(lane_bytes=e["lane_bytes"], mode=e["mode"], pos32=pos32,
                                     sentinel=e.get("sentinel", 0), bitmap=e.get("bitmap", 0))
            else:
                q, alpha = hi.paper_q_alpha(s, m)
                opts = hc.SearchOpts(pos32=pos32)
            filters = []
            for x in pats:
                f = hc.hc_preprocess(x, q, alpha)
                f.to_device()
                filters.append(f)
            out[(s, m)] = (pats, filters, q, alpha, opts)
        return out

    cells = make_cells(args.params)
    paper_cells = make_cells("paper") if args.params == "tuned" else None
    cap = 1 << 27
    pos = torch.empty(cap, dtype=torch.int64 if args.pos64 else torch.int32, device=dev)
    ncell = len(cells)
    counts = torch.zeros((ncell, args.patterns), dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    keys = list(cells.keys())

    def one_step(cell_events=None, which=None):
        which = cells if which is None else which
        for ci, key in enumerate(keys):
            pats, filters, q, alpha, opts = which[key]
            y = texts[key[0]]
            if cell_events is not None:
                cell_events[ci][0].record(stream)
            for pi, f in enumerate(filters):
                hc.hc_search_ex(f, y, pos, counts[ci, pi:pi + 1], opts, cap=cap, stream=stream)
            if cell_events is not None:
                cell_events[ci][1].record(stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    stream.synchronize()
    hc.hc_check_status(stream)
    cnt = counts.cpu().numpy()
    if cnt.max() > cap:
        raise RuntimeError("position buffer too small for this workload")

    ev = lambda: torch.cuda.Event(enable_timing=True)
    step_ev = [[ev(), ev()] for _ in range(args.steps)]
    # the timed step is one CUDA graph of all its searches (captured once,
    # replayed): the device runs them back to back whatever the host does
    # meanwhile (an enqueue loop in Python can stall long enough to drain the
    # launch queue); per-cell times come from events inside the graph
    def graph_ev():
        # recorded by a node of the graph: an external event, to be timed
        try:
            return torch.cuda.Event(enable_timing=True, external=True)
        except TypeError:
            return None
    graph_cell_ev = [[graph_ev(), graph_ev()] for _ in range(ncell)]
    if any(e is None for pair in graph_cell_ev for e in pair):
        graph_cell_ev = None
    graph = None
    launches_per_step = None
    if not args.eager:
        graph = torch.cuda.CUDAGraph()
        l0 = hc.hc_kernel_launches()
        with torch.cuda.graph(graph, stream=stream):
            one_step(graph_cell_ev)
        launches_per_step = hc.hc_kernel_launches() - l0
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                graph.replay()
        stream.synchronize()
        hc.hc_check_status(stream)
    cell_ev = [[[ev(), ev()] for _ in range(ncell)] for _ in range(args.steps)] if args.eager else None

    sampler = ClockSampler(local_rank, interval_ms=max(args.clock_ms, 1), enabled=args.clock_ms > 0)
    launches0 = hc.hc_kernel_launches()
    # the host enqueues the searches; a garbage-collection pause long enough
    # to drain the launch queue would leave the GPU idle inside the timed
    # region, so the collector is off until the measurements are taken
    gc.collect()
    gc.disable()
    barrier()
    sampler.start()
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("hc_timed_steps")   # profilers can select the timed region
    for k in range(args.steps):
        step_ev[k][0].record(stream)
        with torch.cuda.stream(stream):
            if graph is not None:
                graph.replay()
            else:
                one_step(cell_ev[k])
        step_ev[k][1].record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    launches = (hc.hc_kernel_launches() - launches0 if graph is None
                else launches_per_step * args.steps)
    hc.hc_check_status(stream)
    # per-kernel durations: the same steps again with the library's event
    # timing on (an event between the scan and the emit kernel of a search
    # turns off their programmatic overlap, so these steps are not the ones
    # whose time gives `value`)
    hc.hc_timing_report(reset=True)
    hc.hc_timing_enable(True)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            one_step()
    stream.synchronize()
    hc.hc_timing_enable(False)
    kernel_times = hc.hc_timing_report(reset=True)   # {family: (ms, launches)}
    hc.hc_check_status(stream)
    gc.enable()
    counts_tuned = counts.clone()
    paper = None
    if paper_cells is not None:
        # the same sweep on the paper's (q, alpha) (Tables 1-3), for comparison
        pgraph = None
        if not args.eager:
            pgraph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(pgraph, stream=stream):
                one_step(which=paper_cells)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                pgraph.replay() if pgraph is not None else one_step(which=paper_cells)
        gc.collect()
        gc.disable()
        barrier()
        pe0, pe1 = ev(), ev()
        pe0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                pgraph.replay() if pgraph is not None else one_step(which=paper_cells)
        pe1.record(stream)
        barrier()
        gc.enable()
        hc.hc_check_status(stream)
        p_s, p_bytes = combine_ranks(pe0.elapsed_time(pe1) / 1e3,
                                     sum(texts[s].numel() * args.patterns for (s, m) in keys) * args.steps,
                                     dist, dev)
        paper = {"value": round(p_bytes / p_s / GB, 2), "unit": UNIT,
                 "counts_equal": bool(torch.equal(counts, counts_tuned))}
        counts.copy_(counts_tuned)
    step_ms = float(sum(e[0].elapsed_time(e[1]) for e in step_ev))
    if graph is not None and graph_cell_ev is not None:   # the last replay's cell times, for all steps
        cell_ms = np.array([graph_cell_ev[ci][0].elapsed_time(graph_cell_ev[ci][1]) * args.steps
                            for ci in range(ncell)])
    elif graph is not None:   # no timed events inside graphs: the step time split evenly
        cell_ms = np.full(ncell, step_ms / ncell)
    else:
        cell_ms = np.array([sum(cell_ev[k][ci][0].elapsed_time(cell_ev[k][ci][1])
                                for k in range(args.steps)) for ci in range(ncell)])

    text_bytes_step = sum(texts[s].numel() * args.patterns for (s, m) in keys)
    step_s_max, job_bytes = combine_ranks(step_ms / 1e3, text_bytes_step * args.steps, dist, dev)
    value = job_bytes / step_s_max / GB
    ms_per_step = step_s_max * 1e3 / args.steps

    # algorithmic bytes per kernel family (per step): the scan kernels read
    # the text once and spill 4 bytes per occurrence; the emit kernel reads
    # those 4 and writes the position (4 or 8 bytes).  In the dense scan's
    # bitmap form the scan writes one bit per window instead and the emit
    # reads those bits back.
    cnt = counts.cpu().numpy()
    fam_bytes = {}
    per_cell = {}
    for ci, (s, m) in enumerate(keys):
        pats, filters, q, alpha, opts = cells[(s, m)]
        n = texts[s].numel()
        occ = float(cnt[ci].sum())
        fam = scan_family(m, q, opts.mode if opts is not None else 0)
        if fam == "scan_dense" and dense_single_pass(opts, m):
            # one kernel reads the text and writes each position once
            fam_bytes[fam] = fam_bytes.get(fam, 0.0) + n * args.patterns + pos_bytes * occ
        elif fam == "scan_dense" and getattr(opts, "bitmap", 0) == 1:
            bits = (n - m + 1) / 8.0 * args.patterns
            fam_bytes[fam] = fam_bytes.get(fam, 0.0) + n * args.patterns + bits
            fam_bytes["emit"] = fam_bytes.get("emit", 0.0) + bits + pos_bytes * occ
        else:
            fam_bytes[fam] = fam_bytes.get(fam, 0.0) + n * args.patterns + 4 * occ
            fam_bytes["emit"] = fam_bytes.get("emit", 0.0) + (4 + pos_bytes) * occ
        cell_s = cell_ms[ci] / 1e3
        # algorithmic DRAM bytes of the cell's searches: the text once (every
        # byte is read when the whole text is staged; direct-mode cells read
        # less) and each position written once.  The spill region's write and
        # read (8 bytes per occurrence), or the bitmap form's bits, are this
        # implementation's overhead and are not counted.
        alg = (n * args.patterns + pos_bytes * occ) * args.steps
        per_cell[f"s{s}_m{m}"] = {
            "GBps": round(n * args.patterns * args.steps / cell_s / GB, 1),
            "kernel": fam, "q": q, "alpha": alpha,
            "lane_bytes": opts.lane_bytes if opts is not None else 0,
            "form": ("bitmap" if getattr(opts, "bitmap", 0) == 1 else
                     "sentinel" if getattr(opts, "sentinel", 0) == 1 else "plain"),
            "occ_per_pattern": float(cnt[ci].mean()),
            "hbm_frac": round(alg / cell_s / GB / measured_peaks()[0], 3) if fam != "scan_direct" else None,
            "hbm_bytes": "text + positions" if fam != "scan_direct" else None,
        }
    # direct-scan cells: their DRAM bytes from the committed ncu record of
    # the same launch (a fraction of the text; the positions added)
    for ci, (s, m) in enumerate(keys):
        pats, filters, q, alpha, opts = cells[(s, m)]
        name = f"s{s}_m{m}"
        if per_cell[name]["kernel"] != "scan_direct":
            continue
        dram = recorded_cell_traffic(name, q, alpha, opts.lane_bytes if opts is not None else 0,
                                     opts.mode if opts is not None else 0, args.workload)
        if dram is not None:
            occ = float(cnt[ci].sum())
            byts = (dram * args.patterns + pos_bytes * occ) * args.steps
            per_cell[name]["hbm_frac"] = round(byts / (cell_ms[ci] / 1e3) / GB / measured_peaks()[0], 3)
            per_cell[name]["hbm_bytes"] = "ncu DRAM bytes of the scan (profiles/traffic.json) + positions"
    dominant = max(kernel_times, key=lambda k: kernel_times[k][0])
    dom_ms, dom_launches = kernel_times[dominant]
    achieved = fam_bytes.get(dominant, 0.0) * args.steps / (dom_ms / 1e3) / GB if dom_ms else 0.0
    peak, peak_kind = measured_peaks()
    traffic, traffic_rec = recorded_traffic(dominant, args.workload)

    line = {
        "metric": metric_for(args), "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": workload_config(args),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": f"hc_{dominant}", "launches": dom_launches,
                     "avg_launch_us": round(dom_ms * 1e3 / max(dom_launches, 1), 2),
                     "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel_timing": "library CUDA events on the launching stream, over the same "
                                      "steps run again right after the timed region",
                     "traffic_case": (None if traffic_rec is None else
                                      {"case": traffic_rec["case"],
                                       "algorithmic_bytes": traffic_rec["algorithmic_bytes_per_launch"],
                                       "summary": traffic_rec["summary"]})},
        "kernel_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in kernel_times.items() if v[1]},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cells": per_cell,
        "wall_s_timed": round(wall, 3),
    }
    small = [(k, v["hbm_frac"]) for k, v in per_cell.items()
             if int(k.split("_m")[1]) <= 32 and v["hbm_frac"] is not None]
    if small:
        fr = sorted(f for _, f in small)
        line["m_le_32"] = {"cells": len(fr), "at_or_above_0.60": sum(1 for f in fr if f >= 0.60),
                           "median_hbm_frac": fr[len(fr) // 2], "min": fr[0], "max": fr[-1],
                           "note": f"per cell: algorithmic bytes of its searches (text + {pos_bytes} per "
                                   "occurrence) / its device time, of measured HBM"}
    if paper is not None:
        line["paper_params"] = paper
        line["tune_s"] = round(tune_s, 2)
        line["config"]["tuner_table"] = tuner_source
    if args.workload == "skewed":
        line["config"]["sigma_eff"] = {str(s): round(skew_sigma_eff(texts_np[s]), 2) for s in sigmas}
        line["config"]["tuner_sigma"] = {str(s): v for s, v in tune_sigma.items()}

    # ---- end to end through the synchronous C-ABI call, host buffers
    if not args.no_e2e:
        line["e2e"] = e2e_step(args, hc, torch, dev, texts_np, cells, keys, stream, dist,
                               expect=counts_tuned.cpu().numpy(), pos_bytes=pos_bytes)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(texts_np, {k: v[0] for k, v in cells.items()},
                                            args.cpu_seconds, os.cpu_count() or 1)
        # the paper's own setting: one core
        one = cpu_baseline(texts_np, {k: v[0] for k, v in cells.items()}, args.cpu_seconds / 3, 1)
        line["cpu_baseline"]["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
    for key in keys:
        for f in cells[key][1]:
            f.free()
        if paper_cells is not None:
            for f in paper_cells[key][1]:
                f.free()
    if tuner is not None:
        tuner.free()
    return line if rank == 0 else None


BATCH_TUNE_MS = (4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512)


def run_batched(args, rank, world, local_rank):
    """The batched workload: batch_queries(4096) -- n log-uniform 4 KiB to
    64 MiB, m log-uniform 4 to 512, sigma from {4, 20}, each pattern copied
    from its own text.  The batched tuner's table is the stored GB300 one
    (else calibrated first: sigma in {4, 20}, m on a log grid from 4 to 512,
    64 MiB calibration texts; untimed), then one batch with every query's
    (q, alpha) from the tuner (alphabet size measured from each text on the
    device; launch options automatic) runs as a CUDA graph replay.
    Compared with the same batch on the paper's (q, alpha) and with one plain
    hc_search_async launch per query (host-built filters, tuned q, alpha).
    Reports text GB/s (sum of n over device time) of each and the ratios."""
    import torch
    import paper_2310_15711_gb300 as hc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    hc.build()
    hc.lib()
    qrs = hi.batch_queries(args.batch_queries, seed=4)
    offs, total = [], 0
    for qr in qrs:
        offs.append(total)
        total += (qr.n + 15) // 16 * 16
    ybuf = torch.empty(total, dtype=torch.uint8, device=dev)
    host_x = []
    caps = [int(2 * qr.n / float(qr.sigma) ** min(qr.m, 30)) + 64 for qr in qrs]
    pofs = np.concatenate([[0], np.cumsum(caps)])
    pos = {k: torch.empty(int(pofs[-1]), dtype=torch.int64, device=dev) for k in ("tuned", "paper", "plain")}
    counts = {k: torch.zeros(len(qrs), dtype=torch.int64, device=dev) for k in ("tuned", "paper", "plain")}
    xs = []
    for i, qr in enumerate(qrs):
        y = ybuf[offs[i]:offs[i] + qr.n]
        y.copy_(hi.device_uniform_text(qr.n, qr.sigma, qr.text_seed, dev))
        po = int(np.random.default_rng(qr.pattern_seed).integers(0, qr.n - qr.m + 1))
        xs.append(y[po:po + qr.m].clone())
        host_x.append(xs[-1].cpu().numpy())
    text_bytes = float(sum(qr.n for qr in qrs))
    stream = torch.cuda.Stream(device=dev)

    def queries(kind):
        out = []
        for i, qr in enumerate(qrs):
            d = dict(x_dev=xs[i], y_dev=ybuf[offs[i]:offs[i] + qr.n],
                     pos_dev=pos[kind][pofs[i]:pofs[i + 1]], count_dev=counts[kind][i:i + 1])
            if kind == "paper":
                d.update(q=qr.q, alpha=qr.alpha)
            else:
                d.update(q=0, sigma=0)       # tuned; alphabet size measured from the text
            out.append(d)
        return out

    # the batched tuner's table: the stored GB300 one (the calibration's
    # choices vary from run to run, and with them the batch's rate), else
    # calibrated here (saved to --tuner-table when given)
    tuner = hc.HCTuner()
    t0 = time.perf_counter()
    table = getattr(args, "tuner_table", "") or stored_tuner_table(
        "batched", torch.cuda.get_device_name(dev), getattr(args, "retune", False))
    if table and os.path.exists(table):
        tuner.load(table)
        tuner_source = table
    else:
        with torch.cuda.stream(stream):
            tuner.calibrate([4, 20], BATCH_TUNE_MS, text_bytes=args.tune_text_bytes, seed=11, stream=stream)
        stream.synchronize()
        if getattr(args, "tuner_table", ""):
            tuner.save(args.tuner_table)
        tuner_source = "calibrated in this run"
    tune_s = time.perf_counter() - t0
    ev = lambda: torch.cuda.Event(enable_timing=True)

    launches_per_run = {}

    def time_batch(b):
        l0 = hc.hc_kernel_launches()
        with torch.cuda.stream(stream):
            b.run(stream=stream)
        stream.synchronize()
        # preprocessing, one scan per occupancy class of the batch, emit
        launches_per_run[id(b)] = hc.hc_kernel_launches() - l0
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.run(stream=stream)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g.replay()
            e0, e1 = ev(), ev()
            e0.record(stream)
            for _ in range(args.steps):
                g.replay()
            e1.record(stream)
        stream.synchronize()
        hc.hc_check_status(stream)
        return e0.elapsed_time(e1) / args.steps / 1e3

    launches0 = hc.hc_kernel_launches()
    bt = hc.hc_batch_create_tuned(queries("tuned"), tuner)
    # clocks over the timed replays of both batches and the plain launches
    sampler = ClockSampler(local_rank, interval_ms=max(min(args.clock_ms, 50), 1), enabled=args.clock_ms > 0)
    sampler.start()
    t_batch = time_batch(bt)
    tuned_params = [bt.params(i) for i in range(len(qrs))]
    bp = hc.hc_batch_create(queries("paper"))
    t_paper = time_batch(bp)

    filters = []
    for i, qr in enumerate(qrs):
        f = hc.hc_preprocess(host_x[i], tuned_params[i]["q"], tuned_params[i]["alpha"])
        f.to_device()
        filters.append(f)

    def plain_pass():
        for i, qr in enumerate(qrs):
            hc.hc_search_async(filters[i], ybuf[offs[i]:offs[i] + qr.n], pos["plain"][pofs[i]:pofs[i + 1]],
                               counts["plain"][i:i + 1], stream=stream)

    # the plain arm as the batch is timed: all its launches captured in one
    # CUDA graph and replayed (the device runs them back to back, whatever
    # the host does); the eager enqueue loop is reported beside it
    with torch.cuda.stream(stream):
        plain_pass()
    stream.synchronize()
    g_plain = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_plain, stream=stream):
        plain_pass()
    nplain = max(1, args.steps // 2)
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            g_plain.replay()
        e2, e3 = ev(), ev()
        e2.record(stream)
        for _ in range(nplain):
            g_plain.replay()
        e3.record(stream)
        stream.synchronize()
        e4, e5 = ev(), ev()
        e4.record(stream)
        for _ in range(nplain):
            plain_pass()
        e5.record(stream)
    stream.synchronize()
    clocks = sampler.stop()
    hc.hc_check_status(stream)
    del g_plain
    t_plain = e2.elapsed_time(e3) / nplain / 1e3
    t_plain_eager = e4.elapsed_time(e5) / nplain / 1e3
    same = bool(torch.equal(counts["tuned"], counts["plain"]) and torch.equal(counts["tuned"], counts["paper"]))
    nq_changed = sum(1 for i, qr in enumerate(qrs)
                     if (tuned_params[i]["q"], tuned_params[i]["alpha"]) != (qr.q, qr.alpha))
    line = {
        "metric": "batched HC: text GB/s (device-timed, graph replay)",
        "value": round(text_bytes / t_batch / GB, 2), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_batch * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "batched HC", "queries": len(qrs), "text_bytes": int(text_bytes),
                   "n": "log-uniform 4 KiB .. 64 MiB", "m": "log-uniform 4 .. 512",
                   "sigma": "{4, 20}", "q_alpha": "autotuned per (measured sigma, m)",
                   "tuner_table": tuner_source,
                   "l2": "27 GB of texts, far larger than L2; no flush"},
        "queries_per_s": round(len(qrs) / t_batch, 1),
        "paper_params_GBps": round(text_bytes / t_paper / GB, 2),
        "tuned_vs_paper": round(t_paper / t_batch, 3),
        "queries_retuned": nq_changed,
        "plain_launch_GBps": round(text_bytes / t_plain / GB, 2),
        "plain_launch_ms": round(t_plain * 1e3, 3),
        "plain_launch": "one hc_search_async per query, all captured in one CUDA graph and replayed",
        "speedup_vs_plain": round(t_plain / t_batch, 3),
        "plain_eager_GBps": round(text_bytes / t_plain_eager / GB, 2),
        "speedup_vs_plain_eager": round(t_plain_eager / t_batch, 3),
        "counts_equal": same,
        "tune_s": round(tune_s, 2),
        "tuner": tuner.entries(),
        "batch_info": bt.info(),
        "gpu_launches_per_step": launches_per_run[id(bt)],
        "gpu_launches": launches_per_run[id(bt)] * args.steps,
        "library_launches_total": hc.hc_kernel_launches() - launches0,
        "clocks": clocks,
    }
    bt.destroy()
    bp.destroy()
    tuner.free()
    for f in filters:
        f.free()
    return line


SERVED_TUNE_MS = (2, 4, 8, 16, 32, 64, 128, 256, 512, 1024)


def _pct(v, p):
    return float(np.percentile(np.asarray(v, dtype=np.float64), p)) if len(v) else None


def run_served(args, rank, world, local_rank):
    """The served workload: 64 device-resident texts (n log-uniform 1 KiB to
    16 MiB, sigma from {4, 20, 95}), Poisson request streams at 1k, 10k and
    50k requests/s (m log-uniform 2 to 1024, each pattern copied from its
    text), replayed natively into an hc_server (continuous batching, 32 GiB
    admission, tuned parameters) and into a plain server (one search launch
    per request, same parameters), each load repeated --served-reps times
    per server in alternating order.  Reports per load p50/p99 latency over
    the pooled repetitions (from the scheduled arrival to the result on the
    host) and each repetition's p99, achieved requests/s and aggregate text
    GB/s (sum of n over the spans from first arrival to last result), and
    whether every count matches between the two."""
    import torch
    import paper_2310_15711_gb300 as hc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    hc.build()
    hc.lib()
    texts = hi.served_texts(64)
    ydev = [hi.device_uniform_text(n, sigma, seed, dev) for n, sigma, seed in texts]
    yhost = [y.cpu().numpy() for y in ydev]
    tuner = hc.HCTuner()
    t0 = time.perf_counter()
    tuner.calibrate([4, 20, 95], SERVED_TUNE_MS, text_bytes=16 << 20, seed=12)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    loads = []
    sampler = ClockSampler(local_rank, interval_ms=max(args.clock_ms, 1), enabled=args.clock_ms > 0)
    sampler.start()
    # both servers live side by side (texts resident in each); each load runs
    # `reps` times per server, the order alternating, and the latencies of
    # all repetitions are pooled, so that a slow moment of the host does not
    # fall on one server only
    servers = {}
    for plain in (0, 1):
        srv = hc.HCServer(hc.ServerConfig(plain=plain), tuner)
        tids = [srv.add_text(y, sigma=texts[i][1]) for i, y in enumerate(ydev)]
        servers[plain] = (srv, tids)

    def run_stream(plain, rq, arrivals, count):
        srv, _ = servers[plain]
        while srv.poll(65536, positions=False):
            pass
        l0 = hc.hc_kernel_launches()
        ids = srv.replay(rq, arrivals)
        srv.drain()
        res = []
        while len(res) < count:
            res += srv.poll(65536, wait_us=100_000, positions=False)
        launches = hc.hc_kernel_launches() - l0
        pos = {rid: k for k, rid in enumerate(ids)}
        span = (max(r["done_ns"] for r in res) - min(r["submit_ns"] for r in res)) / 1e9
        return res, pos, span, launches

    reps = max(1, args.served_reps)
    for rate in args.served_rates:
        count = max(200, int(rate * args.served_seconds))
        stream = hi.served_requests(texts, count, float(rate), seed=6 + rate)
        arrivals = [a for a, _, _, _ in stream]
        entry = {"offered_req_per_s": rate, "requests": count, "repetitions": reps}
        counts, acc = {}, {0: None, 1: None}
        for plain in (0, 1):   # warm-up (untimed): the first 500 requests, back to back
            tids = servers[plain][1]
            rq = [(tids[ti], yhost[ti][off:off + m]) for _, ti, m, off in stream]
            run_stream(plain, rq[:500], [0.0] * min(500, len(rq)), min(500, len(rq)))
        for rep in range(reps):
            for plain in ((0, 1) if rep % 2 == 0 else (1, 0)):
                tids = servers[plain][1]
                rq = [(tids[ti], yhost[ti][off:off + m]) for _, ti, m, off in stream]
                res, pos, span, launches = run_stream(plain, rq, arrivals, count)
                a = acc[plain] or {"lat": [], "span": 0.0, "bytes": 0, "batches": 0, "max_batch": 0,
                                   "errors": 0, "launches": 0, "p99": []}
                lat = [(r["done_ns"] - r["submit_ns"]) / 1e3 for r in res]
                a["lat"] += lat
                a["p99"].append(round(_pct(lat, 99), 1))
                a["span"] += span
                a["bytes"] += sum(texts[stream[pos[r["id"]]][1]][0] for r in res)
                a["batches"] += len({r["batch"] for r in res})
                a["max_batch"] = max(a["max_batch"], max(r["batch_size"] for r in res))
                a["errors"] += sum(1 for r in res if r["status"] not in (hc.HC_OK, hc.HC_ERR_CAPACITY))
                a["launches"] += launches
                acc[plain] = a
                cnt = {pos[r["id"]]: r["count"] for r in res}
                if plain in counts and counts[plain] != cnt:
                    counts[plain] = None          # a repetition disagreed with the first
                else:
                    counts.setdefault(plain, cnt)
        for plain in (0, 1):
            a = acc[plain]
            st = servers[plain][0].stats()
            entry["plain" if plain else "batched"] = {
                "p50_us": round(_pct(a["lat"], 50), 1),
                "p99_us": float(np.median(a["p99"])),
                "p99_us_pooled": round(_pct(a["lat"], 99), 1),
                "p99_us_per_rep": a["p99"], "mean_us": round(float(np.mean(a["lat"])), 1),
                "achieved_req_per_s": round(count * reps / a["span"], 1),
                "GBps": round(a["bytes"] / a["span"] / GB, 3),
                "batches": a["batches"], "max_batch": a["max_batch"],
                "mean_batch": round(count * reps / max(a["batches"], 1), 2),
                "peak_admitted_MiB": round(st["peak_inflight_bytes"] / 2 ** 20, 2),
                "errors": a["errors"], "gpu_launches": a["launches"],
            }
        entry["counts_equal"] = counts.get(0) is not None and counts.get(0) == counts.get(1)
        entry["p99_ratio_plain_over_batched"] = round(
            entry["plain"]["p99_us"] / max(entry["batched"]["p99_us"], 1e-9), 3)
        loads.append(entry)
    # saturation: a backlog of requests submitted at once, drained as fast as
    # each server can (capacity in requests/s and text GB/s)
    sat = {}
    nsat = args.served_backlog
    stream = hi.served_requests(texts, nsat, 1e9, seed=99)
    sat_counts = {}
    for plain in (0, 1):
        tids = servers[plain][1]
        rq = [(tids[ti], yhost[ti][off:off + m]) for _, ti, m, off in stream]
        run_stream(plain, rq[:500], [0.0] * min(500, len(rq)), min(500, len(rq)))
        res, pos, span, _ = run_stream(plain, rq, [0.0] * len(rq), nsat)
        nbytes = sum(texts[stream[pos[r["id"]]][1]][0] for r in res)
        sat_counts[plain] = {pos[r["id"]]: r["count"] for r in res}
        sat["plain" if plain else "batched"] = {
            "req_per_s": round(nsat / span, 1), "GBps": round(nbytes / span / GB, 3),
            "mean_batch": round(nsat / max(len({r["batch"] for r in res}), 1), 2)}
    for plain in (0, 1):
        servers[plain][0].destroy()
    sat["requests"] = nsat
    sat["speedup_vs_plain"] = round(sat["batched"]["req_per_s"] / sat["plain"]["req_per_s"], 3)
    sat["counts_equal"] = sat_counts[0] == sat_counts[1]
    clocks = sampler.stop()
    top = loads[-1]
    line = {
        "metric": "served HC: aggregate text GB/s at the highest offered load (p50/p99 latency per load)",
        "value": top["batched"]["GBps"], "unit": UNIT, "n_gpus": 1,
        "steps": len(loads), "warmup": 0, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "served HC", "texts": len(texts),
                   "text_n": "log-uniform 1 KiB .. 16 MiB", "sigma": "{4, 20, 95}",
                   "m": "log-uniform 2 .. 1024", "arrivals": "Poisson",
                   "offered_req_per_s": list(args.served_rates), "seconds_per_load": args.served_seconds,
                   "admission_GiB": 32, "q_alpha": "autotuned (sigma in {4, 20, 95}, m 2 .. 1024)",
                   "latency": "scheduled arrival -> result copied on the host",
                   "p99": "median over the repetitions of each repetition's p99 (a host stall of tens of "
                          "ms in one repetition moves a pooled p99 by orders of magnitude; the pooled "
                          "figure is p99_us_pooled)"},
        "p50_us": top["batched"]["p50_us"], "p99_us": top["batched"]["p99_us"],
        "loads": loads, "saturation": sat, "tune_s": round(tune_s, 2),
        "gpu_launches": int(sum(ld["batched"]["gpu_launches"] for ld in loads)),
        "clocks": clocks,
    }
    tuner.free()
    return line


def combine_ranks(seconds, units, dist=None, device=None):
    """Whole-job figures of a multi-rank run: the maximum of the ranks' times
    and the sum of the units they processed (identity on one rank).  Every
    rank must call it; with NCCL the tensors live on `device`."""
    if dist is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def e2e_step(args, hc, torch, dev, texts_np, cells, keys, stream, dist=None, expect=None, pos_bytes=8):
    """One sweep step end to end through the C ABI with host buffers: per
    sigma the text is copied from pinned host memory to the device, then every
    pattern of every cell is searched (hc_search_ex, stream-ordered) and each
    search's positions and count are written by the kernels straight into
    mapped host memory (hc_mapped_alloc: over NVLink-C2C on a Grace-Blackwell
    node, no copy step).  The filters are built before the timed region, as a
    user reuses them across texts.  A timed step ends with the stream
    synchronised and the counts read on the host.

    Two forms of the same calls are timed: enqueued one by one from Python
    (`eager`), and captured once into a CUDA graph -- the copies from pinned
    memory included -- and replayed (the headline: what a user repeating a
    fixed set of searches does; the enqueue loop costs host time per call).
    One untimed eager step comes first (first-touch costs)."""
    pinned = {s: torch.from_numpy(t).pin_memory() for s, t in texts_np.items()}
    y_dev = torch.empty(max(t.numel() for t in pinned.values()), dtype=torch.uint8, device=dev)
    cap = 1 << 27                    # positions (of pos_bytes each)
    nsearch = sum(len(cells[k][1]) for k in keys)
    host_pos = hc.MappedBuffer(cap * pos_bytes // 8)
    host_cnt = hc.MappedBuffer(nsearch)

    def enqueue():
        i = h2d = text_bytes = 0
        for s in sorted(pinned):
            n = pinned[s].numel()
            y_dev[:n].copy_(pinned[s], non_blocking=True)
            h2d += n
            for key in keys:
                if key[0] != s:
                    continue
                pats, filters, q, alpha, opts = cells[key]
                for f in filters:
                    hc.hc_search_ex(f, y_dev[:n], host_pos.view(), host_cnt.view(i, 1), opts,
                                    cap=cap, stream=stream)
                    i += 1
                    text_bytes += n
        return h2d, text_bytes

    def timed(run):
        host_cnt.array()[:] = -1
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            sizes = run()
        stream.synchronize()
        counts = host_cnt.array().copy()
        dt = time.perf_counter() - t0
        hc.hc_check_status(stream)
        return dt, sizes, counts

    timed(enqueue)                                   # untimed warm-up
    dt_e, (h2d, text_bytes), counts_e = timed(enqueue)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        enqueue()
    timed(lambda: graph.replay())                    # untimed first replay
    reps = []
    for _ in range(2):
        dt_g, _, counts_g = timed(lambda: graph.replay())
        reps.append(dt_g)
    dt_g = sum(reps) / len(reps)
    del graph
    d2h = int(sum(pos_bytes * min(int(c), cap) + 8 for c in counts_g))
    same = None if expect is None else bool(np.array_equal(counts_g, expect.reshape(-1)) and
                                            np.array_equal(counts_e, expect.reshape(-1)))
    host_pos.free()
    host_cnt.free()
    dt_g, total_bytes = combine_ranks(dt_g, text_bytes, dist, dev)
    dt_e, _ = combine_ranks(dt_e, text_bytes, dist, dev)
    return {"value": round(total_bytes / dt_g / GB, 2), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h, "counts_equal": same,
            "ms_per_step": round(dt_g * 1e3, 1), "replays": len(reps), "replay_ms": [round(r * 1e3, 1) for r in reps],
            "eager": {"value": round(total_bytes / dt_e / GB, 2), "ms_per_step": round(dt_e * 1e3, 1)},
            "api": "hc_search_ex per pattern (stream-ordered), the step's calls captured once in a CUDA graph "
                   "and replayed (eager: enqueued one by one from Python); texts copied from pinned host memory "
                   "inside the step; positions and counts written by the kernels into mapped host memory "
                   "(hc_mapped_alloc); the step ends with the stream synchronised and the counts read"}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        print(json.dumps(run_batched(args, rank, world, local_rank)), flush=True)
        return
    if args.workload == "served":
        print(json.dumps(run_served(args, rank, world, local_rank)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        line = run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None and args.workload == "sweep" and world == 1 and not args.no_extras and not args.cells:
        line.update(other_workloads(args, local_rank))
    if line is not None:
        print(json.dumps(line), flush=True)


def other_workloads(args, local_rank):
    """The skewed, batched and served configurations, measured in the same
    run as the sweep (one GPU): a compact object each, with the clocks seen
    over its own timed region.  Fewer patterns, steps and seconds than their
    own --workload lines take, so that the default run stays within a few
    minutes."""
    import copy
    out = {}
    t0 = time.perf_counter()
    a = copy.copy(args)
    a.workload, a.patterns, a.no_cpu, a.no_e2e = "skewed", args.extra_patterns, True, True
    a.steps, a.warmup, a.tuner_table = max(3, min(args.steps, 5)), 3, ""
    sk = run_gpu(a, 0, 1, local_rank)
    out["skewed"] = {
        "metric": sk["metric"], "value": sk["value"], "unit": sk["unit"],
        "ms_per_step": sk["ms_per_step"], "steps": sk["steps"], "warmup": sk["warmup"],
        "config": sk["config"], "roofline": sk["roofline"], "m_le_32": sk.get("m_le_32"),
        "paper_params": sk.get("paper_params"), "kernel_ms_per_step": sk["kernel_ms_per_step"],
        "gpu_launches": sk["gpu_launches"], "clocks": sk["clocks"],
        "cells": {k: {"GBps": v["GBps"], "kernel": v["kernel"], "hbm_frac": v["hbm_frac"]}
                  for k, v in sk["cells"].items()}}
    a = copy.copy(args)
    a.workload, a.steps, a.warmup, a.tuner_table = "batched", 3, 3, ""
    bt = run_batched(a, 0, 1, local_rank)
    out["batched"] = {k: bt[k] for k in (
        "metric", "value", "unit", "ms_per_step", "steps", "queries_per_s", "paper_params_GBps",
        "plain_launch_GBps", "plain_launch", "speedup_vs_plain", "plain_eager_GBps",
        "speedup_vs_plain_eager", "counts_equal", "gpu_launches", "clocks")}
    out["batched"]["config"] = bt["config"]
    a = copy.copy(args)
    a.workload, a.served_seconds, a.served_backlog = "served", args.extra_served_seconds, 20000
    sv = run_served(a, 0, 1, local_rank)
    out["served"] = {
        "metric": sv["metric"], "value": sv["value"], "unit": sv["unit"],
        "p50_us": sv["p50_us"], "p99_us": sv["p99_us"], "config": sv["config"],
        "loads": [{"offered_req_per_s": ld["offered_req_per_s"], "requests": ld["requests"],
                   "repetitions": ld["repetitions"], "counts_equal": ld["counts_equal"],
                   "batched": {k: ld["batched"][k] for k in ("p50_us", "p99_us", "p99_us_per_rep",
                                                             "p99_us_pooled", "achieved_req_per_s", "GBps",
                                                             "mean_batch", "gpu_launches")},
                   "plain": {k: ld["plain"][k] for k in ("p50_us", "p99_us", "p99_us_per_rep",
                                                         "p99_us_pooled", "achieved_req_per_s", "GBps")}}
                  for ld in sv["loads"]],
        "saturation": sv["saturation"], "gpu_launches": sv["gpu_launches"], "clocks": sv["clocks"]}
    out["other_workloads_wall_s"] = round(time.perf_counter() - t0, 1)
    return out


if __name__ == "__main__":
    main()
