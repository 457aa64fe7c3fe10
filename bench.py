#!/usr/bin/env python3
"""Label propagation throughput on one GB300 (or N replicas under torchrun).

Headline workload (default "rmat27"): the paper-scale single graph, R-MAT
scale 27 with edge factor 14, (a,b,c,d) = (.57,.19,.19,.05), symmetrised,
de-duplicated, self-loops removed, unit weights, int64 offsets (134,217,728
vertices, ~3.7e9 stored entries), drawn on the device and handed to the
library as host CSR.  One step = one run of the whole hot path in the
paper's asynchronous mode with vertex pruning (initialisation, sweeps until
dN/N <= 0.05 or 20 sweeps, labels out).

Metric: LPA edges/s = sum over runs of nnz x sweeps / time.  Every rank runs
the same workload on its own GPU (replicas, no collective on the data path);
value = all ranks' edges / the slowest rank's time.

Also reported on the same line:
  e2e          the same metric through the public C ABI from pinned host
               buffers: graph creation (H2D copy + validation), the run and
               the labels copied back, all inside the timed region;
  roofline     algorithmic bytes of the dominant kernel per launch / its mean
               launch time, from CUDA events around every launch of the
               profiled run path, against the measured HBM copy bandwidth
               (and the same for all sweep kernels together);
  cpu_baseline the single-threaded CPU oracle on a bounded sample of the
               same graph: its first serial sweep over a contiguous range of
               rows (lpa_inputs.row_range_sample);
  extras       R-MAT 22 + the road-like 4096^2 grid in both modes, with the
               paper's multi-core CPU design on the host cores and the
               tolerance / iteration-cap sweep (Sections 4.1.2-4.1.3);
  batched      the 4,096-graph planted-partition batch in one device loop
               against one lpa_run per graph;
  serving      continuous batching at 2,000 req/s with an R-MAT scale 24
               request every 500, against an unbatched FIFO;
  clocks       nvidia-smi samples taken during the timed region.

--impl reference times the CPU oracle (the reference arm of this method) on
the same workload: each step is one oracle sweep over a bounded sample.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LPA edges/s (|E| x iterations / time)"
UNIT = "edges/s"
TAU = 0.05
MAX_ITERS = 20
MODES = ("sync", "async")
# the sweep kernel of each degree bin (the low-degree bin's asynchronous
# passes run k_sweep_small_async)
BIN_KERNELS = ("k_sweep_small", "k_sweep_warp", "k_sweep_rows<128>", "k_sweep_rows<256>", "k_sweep_rows<512>")
HBM_FALLBACK_GBS = 6800.0


def workload(name):
    import lpa_inputs as L
    if name == "rmat22+grid4096":
        return [("rmat22", lambda: L.rmat(22, 16, seed=1)), ("grid4096", lambda: L.road_grid(4096, 4096, seed=1))]
    if name == "rmat21+grid2048":
        return [("rmat21", lambda: L.rmat(21, 16, seed=1)), ("grid2048", lambda: L.road_grid(2048, 2048, seed=1))]
    if name == "rmat27":
        return [("rmat27", lambda: _rmat_device_host(27))]
    if name == "rmat25":
        return [("rmat25", lambda: _rmat_device_host(25))]
    if name == "rmat24":
        return [("rmat24", lambda: _rmat_device_host(24))]
    if name == "planted1e4+grid64":
        return [("planted1e4", lambda: L.planted_partition(seed=1)), ("grid64", lambda: L.road_grid(64, 64, seed=1))]
    raise SystemExit(f"unknown workload {name}")


def _rmat_device_host(scale):
    """R-MAT of the given scale, edge factor 14, drawn on the device
    (lpa_inputs.device) and copied to host arrays, so the run path starts from
    host CSR like the others."""
    import torch
    import lpa_inputs as L
    from lpa_inputs.device import rmat_device
    g = rmat_device(scale, 14, seed=1)
    host = L.Graph(g.off.cpu().numpy(), g.idx.cpu().numpy(), None,
                   {"kind": "rmat", "scale": scale, "edge_factor": 14, "generator": "device"})
    del g
    torch.cuda.empty_cache()
    return host


# modes each workload runs (every other workload: both)
WORKLOAD_MODES = {"rmat27": ("async",), "rmat25": ("async",), "rmat24": ("async",)}

WORKLOAD_TEXT = {
    "rmat22+grid4096": "R-MAT scale 22 edge factor 16 (a,b,c,d=.57,.19,.19,.05; symmetrised, deduplicated, "
                       "no self-loops; unit weights) + 4096x4096 road-like grid (10% edges dropped, 0.1% "
                       "shortcuts, integer weights 1..8); sync and async-with-pruning; tau=0.05, cap 20",
    "rmat21+grid2048": "R-MAT scale 21 + 2048x2048 road-like grid (smaller profiling case of the same "
                       "generators, still larger than L2); sync and async-with-pruning; tau=0.05, cap 20",
    "rmat27": "R-MAT scale 27 edge factor 14 (a,b,c,d=.57,.19,.19,.05; symmetrised, deduplicated, no "
              "self-loops; unit weights; ~3.7e9 entries, int64 offsets; drawn on the device with torch); "
              "asynchronous mode with pruning; tau=0.05, cap 20",
    "rmat25": "R-MAT scale 25 edge factor 14 (the generator and mode of the scale-27 workload at a "
              "quarter of the size: ~0.9e9 entries, a 134 MB label array just above L2; a profiling "
              "case); asynchronous mode with pruning; tau=0.05, cap 20",
    "rmat24": "R-MAT scale 24 edge factor 14 (~0.45e9 entries, a few GB on the device: the case for "
              "multi-pass ncu captures of the scale-27 kernels); asynchronous mode with pruning; tau=0.05, cap 20",
    "planted1e4+grid64": "planted partition 10 x 1000 + 64x64 road-like grid (a seconds-long check of the "
                         "launch path, smaller than L2: not a performance workload); tau=0.05, cap 20",
}


# DRAM bytes (read + write) per launch from one ncu capture of the same
# command (dram__bytes_read.sum + dram__bytes_write.sum over every launch of
# the kernel in one step of the profiled run path), valid only while the
# kernel's sources are unchanged (sha1 of the files below).
TRAFFIC = {
    # R-MAT 27, asynchronous, caller's storage order: 83.1 GB over the six
    # launches of one run (profiles/dram_traffic_rmat27_async.md)
    "k_sweep_rows<512>": {"bytes_per_launch": 13.845e9, "sha1": "65d8471627fce658f1fa91866f02670ef6ea9178",
                          "workload": "rmat27", "order": "caller",
                          "files": ["lpa_sweep_rows.cu", "lpa_device.cuh", "lpa_internal.h"]},
}


def measured_traffic(kernel, args):
    import hashlib
    t = TRAFFIC.get(kernel)
    if not t or t["workload"] != args.workload or t["order"] != args.order:
        return None
    h = hashlib.sha1()
    for f in t["files"]:
        with open(os.path.join(ROOT, "paper_2312_08140_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return t["bytes_per_launch"] if h.hexdigest() == t["sha1"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- oracle arm
def oracle_run(g, mode, max_iters):
    """The oracle's run for a mode string of the library ("sync", "async",
    "sync_full", with "+nonstrict" / "+prune_other"); returns (labels,
    iterations, changed)."""
    import oracle as O
    base, *flags = mode.split("+")
    nonstrict = "nonstrict" in flags
    if base in ("sync", "sync_full"):
        return O.lpa_sync(g.off, g.idx, g.w, TAU, max_iters, nonstrict=nonstrict)
    if "prune_other" in flags:
        return O.lpa_async_ex(g.off, g.idx, g.w, TAU, max_iters, nonstrict=nonstrict, prune_other=True)[:3]
    return O.lpa_async(g.off, g.idx, g.w, TAU, max_iters, nonstrict=nonstrict)


def oracle_sample(graphs, pairs):
    """Times one oracle sweep per (graph, mode) pair; returns (edges, seconds)."""
    edges, secs = 0, 0.0
    for gi, mode in pairs:
        g = graphs[gi]
        t0 = time.perf_counter()
        _, it, _ = oracle_run(g, mode, 1)
        secs += time.perf_counter() - t0
        edges += g.nnz * it
    return edges, secs


def host_cpu():
    """Cores and model of the host that runs the CPU legs."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model Name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "lscpu_model": model}


def oracle_rows_sample(g, mode, v0, entries):
    """One oracle sweep (the first sweep of the mode's run) over the rows of g
    starting at v0 and holding about `entries` entries
    (lpa_inputs.row_range_sample: the rows and their neighbours, relabelled in
    order, the neighbours' rows empty).  Returns (entries scanned, seconds,
    (v0, v1))."""
    import lpa_inputs as L
    sg, v1, _ = L.row_range_sample(g, v0, entries)
    t0 = time.perf_counter()
    oracle_run(sg, mode, 1)
    return sg.nnz, time.perf_counter() - t0, (int(v0), int(v1))


def oracle_rows_baseline(g, mode, target_s=12.0):
    """The oracle on a bounded sample of a graph too large to sweep whole on
    one core: rows from the middle of the id range, sized from a short first
    sample so that the timed sample takes about target_s seconds."""
    v0 = g.n // 3
    e, t, _ = oracle_rows_sample(g, mode, v0, 1 << 22)
    rate = e / max(t, 1e-6)
    want = int(min(max(rate * target_s, 1 << 22), 1 << 30))
    e, t, rows = oracle_rows_sample(g, mode, v0, want)
    return e, t, rows


def workload_modes(args):
    """The mode strings one step runs on each graph of the workload."""
    modes = WORKLOAD_MODES.get(args.workload, MODES)
    if args.tie == "nonstrict":
        modes = tuple(m + "+nonstrict" for m in modes)
    if args.prune == "other":
        modes = tuple(m + "+prune_other" if m.startswith("async") else m for m in modes)
    return modes


def run_config(args, world):
    """The JSON line's config object, the same for both arms."""
    return {"workload": WORKLOAD_TEXT[args.workload], "tie_break": args.tie,
            "storage_order": args.order,
            "async_pruning": "FLPA rule" if args.prune == "other" else "every neighbour",
            "inputs_larger_than_l2": True,
            "parallelism": f"replicas x{world}", "tau": TAU, "max_iters": MAX_ITERS}


def param_sweep(lpa, torch, stream, names, graphs, handles, outs, mode="async", reps=3):
    """Tolerance and iteration-cap sweep per graph class (the paper's ablations
    of Sections 4.1.2-4.1.3): for tau in {0.1, 0.05, 0.01, 1e-5} and cap in
    {10, 20, 50}, sweeps run, device time per run, edges/s, time per stored
    entry and the modularity (Eq. 1) of the labels."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for name, g, h, o in zip(names, graphs, handles, outs):
        for tau in (0.1, 0.05, 0.01, 1e-5):
            for cap in (10, 20, 50):
                info = lpa.lpa_run(h, mode, tau, cap, o, stream, info=True)
                torch.cuda.synchronize()
                ev0.record(stream)
                for _ in range(reps):
                    lpa.lpa_run(h, mode, tau, cap, o, stream, info=False)
                ev1.record(stream)
                torch.cuda.synchronize()
                ms = ev0.elapsed_time(ev1) / reps
                q = lpa.lpa_modularity(h, o)
                rows.append({"graph": name, "mode": mode, "tau": tau, "cap": cap, "iterations": info.iterations,
                             "ms": ms, "edges_per_s": g.nnz * info.iterations / (ms / 1e3),
                             "ns_per_entry": ms * 1e6 / g.nnz, "modularity": q})
    return rows


def cpu_parallel_sample(graphs, modes):
    """The paper's own multi-core CPU design (cpu_parallel: OpenMP dynamic
    chunks, per-thread collision-free tables, 8-bit flags) on the host cores:
    one full run of each (graph, mode) pair of the workload."""
    import cpu_parallel as CP
    edges, secs = 0, 0.0
    for g in graphs:
        for m in modes:
            if "+" in m:
                continue                                   # the CPU design has the strict tie-break only
            t0 = time.perf_counter()
            _, it, _ = CP.run(g.off, g.idx, g.w, m, TAU, MAX_ITERS)
            secs += time.perf_counter() - t0
            edges += g.nnz * it
    if secs == 0.0:
        return None
    return {"value": edges / secs, "unit": UNIT, "cores": CP.threads(), "kind": "paper design, OpenMP",
            "sample": f"one full run of each (graph, mode) pair of the workload ({secs:.1f} s)"}


LARGE_NNZ = 400_000_000       # above this a whole oracle sweep of a graph takes minutes: time row samples
REF_SAMPLE_ENTRIES = 1 << 24  # entries per reference-arm step on a large graph


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    O.build()
    wl = workload(args.workload)
    graphs = [make() for _, make in wl]
    modes = workload_modes(args)
    pairs = [(gi, m) for gi in range(len(graphs)) for m in modes]
    large = any(g.nnz > LARGE_NNZ for g in graphs)
    total = args.warmup + args.steps

    def one(step):
        gi, m = pairs[step % len(pairs)]
        g = graphs[gi]
        if g.nnz > LARGE_NNZ:
            e, t, _ = oracle_rows_sample(g, m, (g.n * (step + 1)) // (total + 1), REF_SAMPLE_ENTRIES)
            return e, t
        return oracle_sample(graphs, [(gi, m)])

    for s in range(args.warmup):
        one(s)
    edges, secs = 0, 0.0
    t_all = time.perf_counter()
    for s in range(args.steps):
        e, t = one(args.warmup + s)
        edges += e
        secs += t
    wall = time.perf_counter() - t_all
    value = edges / secs
    if large:
        sample = (f"each step: the CPU oracle's first sweep over a range of about {REF_SAMPLE_ENTRIES} entries "
                  f"of rows of {[wl[g][0] for g, _ in pairs]} ({[m for _, m in pairs]} mode), the range moving "
                  f"through the vertex ids from step to step (rows and their neighbours relabelled in order)")
    else:
        sample = (f"each step: one CPU-oracle sweep of one (graph, mode) pair, rotating over "
                  f"{[(wl[g][0], m) for g, m in pairs]}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": run_config(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- batched and serving
def batched_sample(lpa, torch, stream, G, reps=5):
    """G graphs of the batched planted-partition distribution (seeds 1000+g):
    one handle and one device loop per run, against one handle and one
    lpa_run per graph on the same stream."""
    import numpy as np
    import lpa_inputs as L
    graphs = [L.batched_sbm_graph(g) for g in range(G)]
    vo, eo, off, _, w = L.pack(graphs)
    idx = np.concatenate([gr.idx for gr in graphs]).astype(np.int32)
    N = int(vo[-1])
    b = lpa.lpa_batch_create(G, vo, eo, off, idx, w, lpa.LPA_HOST_PTRS, stream)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    res = {"graphs": G, "vertices": N, "entries": int(eo[-1])}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for m in MODES:
        infos = lpa.lpa_batch_run(b, G, m, TAU, MAX_ITERS, out, stream, info=True)
        edges = sum(gr.nnz * inf.iterations for gr, inf in zip(graphs, infos))
        for _ in range(2):
            lpa.lpa_batch_run(b, G, m, TAU, MAX_ITERS, out, stream, info=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            lpa.lpa_batch_run(b, G, m, TAU, MAX_ITERS, out, stream, info=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3 / reps
        res[m] = {"batched_graphs_per_s": G / sec, "batched_edges_per_s": edges / sec, "batched_ms": sec * 1e3}
    lpa.lpa_batch_destroy(b)
    handles = [lpa.lpa_graph_create(gr.n, gr.nnz, gr.off, gr.idx, gr.w, lpa.LPA_HOST_PTRS, stream) for gr in graphs]
    outs = [torch.empty(max(gr.n, 1), dtype=torch.int32, device="cuda") for gr in graphs]
    for m in MODES:
        for h, o in zip(handles, outs):
            lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            for h, o in zip(handles, outs):
                lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3 / reps
        res[m]["one_launch_per_graph_graphs_per_s"] = G / sec
        res[m]["speedup_vs_one_launch_per_graph"] = res[m]["batched_graphs_per_s"] / (G / sec)
    for h in handles:
        lpa.lpa_graph_destroy(h)
    return res


def batched_sample_full(lpa, torch, stream, G=4096, reps=3):
    """The full batched workload: 4,096 planted-partition graphs drawn on the
    device (lpa_inputs.device), one handle and one device loop per run, against
    one handle and one lpa_run per graph (handles made from device slices)."""
    import numpy as np
    from lpa_inputs.device import batched_planted_partition_device
    vo, eo, off, idx, w, _ = batched_planted_partition_device(G)
    torch.cuda.empty_cache()
    N = int(vo[-1])
    b = lpa.lpa_batch_create(G, vo, eo, off, idx, w, lpa.LPA_DEVICE_PTRS, stream)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    nnz = np.diff(eo)
    res = {"graphs": G, "vertices": N, "entries": int(eo[-1]), "inputs": "drawn on the device"}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    default_cfg = lpa.lpa_batch_get_config(b)

    def timed(m):
        lpa.lpa_batch_run(b, G, m, TAU, MAX_ITERS, out, stream, info=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            lpa.lpa_batch_run(b, G, m, TAU, MAX_ITERS, out, stream, info=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps

    for m in MODES:
        lpa.lpa_batch_set_config(b, default_cfg)
        infos = lpa.lpa_batch_run(b, G, m, TAU, MAX_ITERS, out, stream, info=True)
        edges = int(sum(int(nnz[k]) * infos[k].iterations for k in range(G)))
        sec = timed(m)
        res[m] = {"batched_graphs_per_s": G / sec, "batched_edges_per_s": edges / sec, "batched_ms": sec * 1e3,
                  "config": default_cfg.as_dict()}
        # the batched autotuner: a search timed on a sampled sub-batch (1/8 of
        # the entries), its pick then timed on the whole batch
        cfg, tinfo = lpa.lpa_batch_autotune(b, m, TAU, MAX_ITERS, 2, 125, stream)
        sec_t = timed(m)
        res[m]["autotuned"] = {"config": cfg.as_dict(), "batched_graphs_per_s": G / sec_t,
                               "batched_ms": sec_t * 1e3, "search_ms": tinfo["search_ms"],
                               "candidates": tinfo["candidates"], "sample_graphs": tinfo["sample_graphs"]}
    lpa.lpa_batch_set_config(b, default_cfg)
    lpa.lpa_batch_destroy(b)
    handles, outs = [], []
    for k in range(G):
        v0, v1, e0, e1 = int(vo[k]), int(vo[k + 1]), int(eo[k]), int(eo[k + 1])
        o = (off[v0:v1 + 1] - e0).contiguous()
        handles.append(lpa.lpa_graph_create(v1 - v0, e1 - e0, o, idx[e0:e1], w[e0:e1], lpa.LPA_DEVICE_PTRS, stream))
        outs.append(torch.empty(max(v1 - v0, 1), dtype=torch.int32, device="cuda"))
    del off, idx, w
    for m in MODES:
        for h, o in zip(handles, outs):
            lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        for h, o in zip(handles, outs):
            lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        res[m]["one_launch_per_graph_graphs_per_s"] = G / sec
        res[m]["speedup_vs_one_launch_per_graph"] = res[m]["batched_graphs_per_s"] / (G / sec)
    for h in handles:
        lpa.lpa_graph_destroy(h)
    torch.cuda.empty_cache()
    return res


def _percentiles(lat):
    import numpy as np
    a = np.asarray(lat) * 1e3
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean())}


def serving_sample(lpa, torch, stream, rate, seconds, pool_size, big=None, big_every=0, seed=1):
    """Poisson arrivals at `rate` req/s for `seconds`, requests drawn from a
    pool of the batched distribution (and `big` every `big_every` requests):
    the continuous-batching server against an unbatched FIFO that creates a
    graph and runs lpa_run for one request at a time."""
    import numpy as np
    import lpa_inputs as L
    rng = np.random.default_rng(seed)

    def pinned(g):    # request buffers in page-locked memory, as a server's receive buffers would be
        pin = lambda a: None if a is None else torch.from_numpy(a).pin_memory().numpy()
        return L.Graph(pin(g.off), pin(g.idx), pin(g.w), g.meta)

    pool = [pinned(L.batched_sbm_graph(g)) for g in range(pool_size)]
    if big is not None:
        big = pinned(big)
    count = int(rate * seconds)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=count))
    picks = rng.integers(0, pool_size, size=count)
    reqs = [(big if (big is not None and big_every and (k + 1) % big_every == 0) else pool[picks[k]])
            for k in range(count)]
    max_n = max(g.n for g in pool)
    max_e = max(g.nnz for g in pool)
    srv = lpa.lpa_serve_create(hbm_budget_bytes=48 << 30, arena_vertices=64 * max_n, arena_entries=64 * max_e,
                               max_slots=256, mode="sync", tolerance=TAU, max_iters=MAX_ITERS,
                               solo_min_entries=(4 * max_e if big is not None else 0))
    t0 = time.perf_counter()
    submit_t, done_t, ticket_of = {}, {}, {}
    submit_s = 0.0
    backlog = list(range(count))
    k_next = 0
    while len(done_t) < count:
        now = time.perf_counter() - t0
        while k_next < count and arrivals[k_next] <= now:
            k_next += 1
        while backlog and backlog[0] < k_next:
            k = backlog[0]
            g = reqs[k]
            ts = time.perf_counter()
            try:
                t = lpa.lpa_serve_submit(srv, g.n, g.nnz, g.off, g.idx, g.w)
                submit_s += time.perf_counter() - ts
            except lpa.LpaError as e:
                if e.status != lpa.LPA_ERR_BUSY:
                    raise
                break
            ticket_of[t] = k
            backlog.pop(0)
        for t in lpa.lpa_serve_poll(srv):
            done_t[ticket_of[t]] = time.perf_counter() - t0
            lpa.lpa_serve_release(srv, t)
        if time.perf_counter() - t0 > seconds * 20 + 60:
            raise RuntimeError("serving sample did not drain")
        time.sleep(0.0002)
    stats = lpa.lpa_serve_stats(srv)
    lpa.lpa_serve_destroy(srv)
    lat = [done_t[k] - arrivals[k] for k in range(count)]
    span = max(done_t.values()) - arrivals[0]
    served = {"requests": count, "offered_req_per_s": rate, "graphs_per_s": count / span,
              "cycles": stats["cycles"], "cycles_per_s": stats["cycles"] / span,
              "submit_ms_mean": 1e3 * submit_s / count, **_percentiles(lat)}
    # unbatched FIFO: one graph handle and one lpa_run per request, in arrival order
    out = torch.empty(max(max(g.n for g in reqs), 1), dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    fifo_done = []
    for k in range(count):
        now = time.perf_counter() - t0
        if now < arrivals[k]:
            time.sleep(arrivals[k] - now)
        g = reqs[k]
        h = lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w, lpa.LPA_HOST_PTRS, stream)
        lpa.lpa_run(h, "sync", TAU, MAX_ITERS, out, stream, info=False)
        lab = out[:g.n].cpu()
        del lab
        lpa.lpa_graph_destroy(h)
        fifo_done.append(time.perf_counter() - t0)
    flat = [fifo_done[k] - arrivals[k] for k in range(count)]
    fifo = {"graphs_per_s": count / (fifo_done[-1] - arrivals[0]), **_percentiles(flat)}
    return {"server": served, "unbatched_fifo": fifo}


# ------------------------------------------------------------------- GPU arm
def reduce_over_ranks(dist, device, slowest, counts):
    """Replicas: the job's time is the slowest rank's and its work the sum of
    every rank's counters.  Returns (max over ranks, [sums])."""
    if dist is None:
        return float(slowest), [float(c) for c in counts]
    import torch
    t = torch.tensor([float(slowest)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(c) for c in counts], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(x) for x in u.tolist()]


def kernel_bytes(prof, wbytes, sync, passes, rows_distinct=False):
    """Algorithmic bytes per sweep-kernel launch from the per-bin counts:
    per scanned vertex 16 B offsets + 4 B own label + 4 B frontier id; per
    scanned entry 4 B index + wbytes weight + 4 B gathered label (none in the
    first synchronous sweep of a graph whose rows repeat no neighbour: its
    labels are still the vertex ids); per changed vertex 4 B label write (+4 B
    changed-list entry in sync mode) and 1 B flag per entry of its row."""
    out = {b: {"bytes": 0.0, "ms": 0.0, "launches": 0} for b in BIN_KERNELS}
    if not prof["iterations"]:
        return out
    # the first sweep scans every vertex with an entry: a bin empty then is
    # statically empty and never launched
    launched = [prof["bin_vertices"][0][bi] > 0 for bi in range(len(BIN_KERNELS))]
    for t in range(min(prof["iterations"], 64)):
        gather = 0 if (sync and rows_distinct and t == 0) else 4
        for bi, b in enumerate(BIN_KERNELS):
            if not launched[bi]:
                continue
            v = prof["bin_vertices"][t][bi]
            e = prof["bin_entries"][t][bi]
            c = prof["bin_changed"][t][bi]
            ce = prof["bin_changed_entries"][t][bi]
            by = v * 24 + e * (4 + wbytes + gather) + c * (8 if sync else 4) + ce
            out[b]["bytes"] += by
            out[b]["ms"] += prof["sweep_ms"][t][bi]
            out[b]["launches"] += passes
    return out


def release(lpa, torch, handles):
    for h in handles:
        lpa.lpa_graph_destroy(h)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    lpa.lpa_release_cached_memory()


def run_extras(lpa, torch, stream, tie, prune, reps=5):
    """R-MAT 22 + the road-like 4096^2 grid in both modes: device
    edges/s per (graph, mode), the paper's multi-core CPU design on the host
    cores, and the tolerance / cap sweep per graph class."""
    args = argparse.Namespace(workload="rmat22+grid4096", tie=tie, prune=prune)
    wl = workload(args.workload)
    graphs = [make() for _, make in wl]
    modes = workload_modes(args)
    handles = [lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w, lpa.LPA_HOST_PTRS, stream) for g in graphs]
    outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = []
    edges_all, ms_all = 0, 0.0
    for (name, _), g, h, o in zip(wl, graphs, handles, outs):
        for m in modes:
            info = lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=True)
            for _ in range(2):
                lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / reps
            edges_all += g.nnz * info.iterations
            ms_all += ms
            runs.append({"graph": name, "mode": m, "n": g.n, "nnz": g.nnz, "iterations": info.iterations,
                         "exit_reason": info.exit_reason, "ms": ms, "edges_per_s": g.nnz * info.iterations / (ms / 1e3),
                         "touched_per_s": info.edges_touched / (ms / 1e3),
                         "modularity": lpa.lpa_modularity(h, o)})
    res = {"workload": WORKLOAD_TEXT[args.workload], "edges_per_s": edges_all / (ms_all / 1e3), "runs": runs,
           "param_sweep": param_sweep(lpa, torch, stream, [n for n, _ in wl], graphs, handles, outs),
           "cpu_parallel": cpu_parallel_sample(graphs, modes)}
    release(lpa, torch, handles)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gvelpa", choices=["gvelpa", "reference"])
    ap.add_argument("--workload", default="rmat27", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true", help="skip the event-timed roofline pass")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the R-MAT 22 + grid runs, the paper's CPU design and the tau / cap sweep")
    ap.add_argument("--batched-graphs", type=int, default=4096,
                    help="4096: the full batch drawn on the device; other N: N host-drawn graphs; 0 skips it")
    ap.add_argument("--serving-requests", type=int, default=10_000, help="0 skips the serving sample")
    ap.add_argument("--serving-big-every", type=int, default=500,
                    help="an R-MAT scale 24 request every this many requests (0: none)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick each graph's degree-bin launch parameters with lpa_autotune (two timed runs per "
                         "candidate) before the warm-up; the search time is reported, not timed")
    ap.add_argument("--order", default="caller", choices=["caller", "degree", "shuffle"],
                    help="storage order of the graphs' vertices (lpa_graph_create flags; labels stay caller ids)")
    ap.add_argument("--profile-only", action="store_true",
                    help="create the workload's graphs, run each mode twice through the host-launched profiled "
                         "path (every kernel a separate launch, as ncu needs) and print the per-bin times")
    ap.add_argument("--tie", default="strict", choices=["strict", "nonstrict"],
                    help="tie-break among the most weighted labels (Section 4.1.5)")
    ap.add_argument("--prune", default="paper", choices=["paper", "other"],
                    help="async pruning: every neighbour of a changed vertex re-marked (Section 4.1.4), or "
                         "only those not already in its new label (FLPA's rule, Section 2)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_2312_08140_gb300 as lpa
    lpa.load()

    wl = workload(args.workload)
    graphs = [make() for _, make in wl]
    modes = workload_modes(args)
    stream = torch.cuda.current_stream()
    order_flag = {"caller": 0, "degree": lpa.LPA_REORDER_DEGREE, "shuffle": lpa.LPA_REORDER_SHUFFLE}[args.order]
    handles = [lpa.lpa_graph_create(g.n, g.nnz, g.off, g.idx, g.w, lpa.LPA_HOST_PTRS | order_flag, stream)
               for g in graphs]
    outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g in graphs]
    tuned, tuned_cfgs = None, [None] * len(graphs)
    if args.autotune:
        tuned = {}
        for gi, ((name, _), h) in enumerate(zip(wl, handles)):
            cfg, info = lpa.lpa_autotune(h, modes[0], TAU, MAX_ITERS, 2, stream)
            tuned_cfgs[gi] = cfg
            tuned[name] = {"config": cfg.as_dict(), "default_ms": round(info["default_ms"], 3),
                           "chosen_ms": round(info["chosen_ms"], 3), "search_ms": round(info["search_ms"], 1),
                           "candidates": info["candidates"]}
            print(json.dumps({"autotune": name, **tuned[name]}), file=sys.stderr, flush=True)
    if args.profile_only:
        # two profiled runs per mode: the first one's times include the lazy
        # loading of each kernel at its first launch
        for (name, _), h, o in zip(wl, handles, outs):
            for m, run in ((m, r) for m in modes for r in range(2)):
                ri, prof = lpa.lpa_run_profiled(h, m, TAU, MAX_ITERS, o, stream)
                p = prof.as_dict()
                print(json.dumps({"graph": name, "mode": m, "run": run, "iterations": ri.iterations,
                                  "bins": list(BIN_KERNELS), "sweep_ms": p["sweep_ms"],
                                  "finish_ms": p["finish_ms"], "bin_vertices": p["bin_vertices"],
                                  "bin_entries": p["bin_entries"]}), flush=True)
        release(lpa, torch, handles)
        return

    def step():
        for h, g, o in zip(handles, graphs, outs):
            for m in modes:
                lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    before = [lpa.lpa_graph_props_get(h) for h in handles]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    after = [lpa.lpa_graph_props_get(h) for h in handles]
    sweeps = [a["sweeps_total"] - b["sweeps_total"] for a, b in zip(after, before)]
    edges = sum(g.nnz * s for g, s in zip(graphs, sweeps))
    touched = sum(a["scanned_total"] - b["scanned_total"] for a, b in zip(after, before))
    launches = sum(a["launches_total"] - b["launches_total"] for a, b in zip(after, before))
    ms, (edges, touched, launches) = reduce_over_ranks(dist, "cuda", ms, [edges, touched, launches])
    value = edges / (ms / 1e3)

    # per-run detail (one run each, with info) for the record
    per_run = []
    for (name, _), h, g, o in zip(wl, handles, graphs, outs):
        for m in modes:
            ri = lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=True)
            per_run.append({"graph": name, "mode": m, "n": g.n, "nnz": g.nnz, "iterations": ri.iterations,
                            "exit_reason": ri.exit_reason, "scanned": ri.edges_touched})

    # e2e through the public API from pinned host memory
    pinned = []
    for g in graphs:
        t_off = torch.from_numpy(g.off).pin_memory()
        t_idx = torch.from_numpy(g.idx).pin_memory()
        t_w = torch.from_numpy(g.w).pin_memory() if g.w is not None else None
        t_lab = torch.empty(g.n, dtype=torch.int32).pin_memory()
        pinned.append((t_off, t_idx, t_w, t_lab))
    h2d = sum(g.off.nbytes + g.idx.nbytes + (g.w.nbytes if g.w is not None else 0) for g in graphs)
    d2h = sum(4 * g.n * len(modes) for g in graphs)

    def e2e_step():
        e = 0
        for g, (t_off, t_idx, t_w, t_lab), o, cfg in zip(graphs, pinned, outs, tuned_cfgs):
            h = lpa.lpa_graph_create(g.n, g.nnz, t_off, t_idx, t_w, lpa.LPA_HOST_PTRS | order_flag, stream)
            if cfg is not None:
                lpa.lpa_graph_set_config(h, cfg)
            for m in modes:
                lpa.lpa_run(h, m, TAU, MAX_ITERS, o, stream, info=False)
                t_lab.copy_(o, non_blocking=True)
            e += g.nnz * lpa.lpa_graph_props_get(h)["sweeps_total"]   # waits for the device
            lpa.lpa_graph_destroy(h)
        return e

    e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_edges = sum(e2e_step() for _ in range(args.e2e_steps))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s, (e2e_edges,) = reduce_over_ranks(dist, "cuda", e2e_s, [e2e_edges])

    # roofline: event-timed profiled runs, same kernels and launch shapes
    roofline, kernels = None, None
    hbm, hbm_kind = peaks()
    if not args.no_profile:
        agg = {}
        for g, h, o in zip(graphs, handles, outs):
            props = lpa.lpa_graph_props_get(h)
            wbytes = props["weight_bytes"]                           # as the sweeps read them
            for m in modes:
                _, prof = lpa.lpa_run_profiled(h, m, TAU, MAX_ITERS, o, stream)
                sync = not m.startswith("async")
                for b, d in kernel_bytes(prof.as_dict(), wbytes, sync, 1 if sync else 2,
                                         props["rows_distinct"]).items():
                    a = agg.setdefault(b, {"bytes": 0.0, "ms": 0.0, "launches": 0})
                    for k in a:
                        a[k] += d[k]
        kernels = {}
        for b, a in agg.items():
            if a["launches"] and a["ms"] > 0:
                kernels[b] = {"launches_per_step": a["launches"], "ms_per_step": a["ms"],
                                           "GB_per_s": a["bytes"] / (a["ms"] / 1e3) / 1e9,
                                           "bytes_per_launch": a["bytes"] / a["launches"]}
        dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
        d = kernels[dom]
        roofline = {"bound": "hbm", "kernel": dom, "achieved": d["GB_per_s"], "peak": hbm, "unit": "GB/s",
                    "frac": d["GB_per_s"] / hbm, "peak_kind": hbm_kind, "traffic": measured_traffic(dom, args),
                    "bytes_per_launch": d["bytes_per_launch"],
                    "mean_launch_ms": d["ms_per_step"] / d["launches_per_step"]}
        if roofline["traffic"]:
            # the DRAM bytes ncu counted per launch, at this run's launch time
            roofline["traffic_GB_per_s"] = roofline["traffic"] / (roofline["mean_launch_ms"] / 1e3) / 1e9
            roofline["traffic_frac"] = roofline["traffic_GB_per_s"] / hbm
        tot_b = sum(a["bytes"] for a in agg.values())
        tot_ms = sum(a["ms"] for a in agg.values())
        if tot_ms > 0:
            roofline["all_sweep_kernels"] = {"achieved": tot_b / (tot_ms / 1e3) / 1e9, "unit": "GB/s",
                                             "frac": tot_b / (tot_ms / 1e3) / 1e9 / hbm,
                                             "bytes_per_step": tot_b, "ms_per_step": tot_ms}

    # the CPU oracle on the host cores: a bounded sample of the same workload
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if any(g.nnz > LARGE_NNZ for g in graphs):
            e_all, s_all, parts = 0, 0.0, []
            for (name, _), g in zip(wl, graphs):
                for m in modes:
                    e, t, rows = oracle_rows_baseline(g, m)
                    e_all += e
                    s_all += t
                    parts.append(f"{name} {m}: rows [{rows[0]}, {rows[1]}), {e} entries, {t:.1f} s")
            cpu = {"value": e_all / s_all, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "the CPU oracle's first sweep over a contiguous range of rows (the rows and their "
                             "neighbours relabelled in order, neighbours' rows empty): " + "; ".join(parts),
                   **host_cpu()}
        else:
            pairs = [(gi, m) for gi in range(len(graphs)) for m in modes]
            e, s_ = oracle_sample(graphs, pairs + pairs)
            cpu = {"value": e / s_, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": "CPU oracle, one sweep of each (graph, mode) pair of the workload, twice "
                             f"({s_:.1f} s of single-thread CPU work)", **host_cpu()}
    cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and sum(g.nnz for g in graphs) <= LARGE_NNZ:
        cpu_par = cpu_parallel_sample(graphs, modes)

    # the headline graphs are freed before the other samples
    del pinned
    release(lpa, torch, handles)
    del graphs, outs
    torch.cuda.empty_cache()

    extras = None
    if args.workload == "rmat27" and not args.no_extras:
        extras = run_extras(lpa, torch, stream, args.tie, args.prune)
    batched = None
    if args.batched_graphs == 4096:
        batched = batched_sample_full(lpa, torch, stream)
    elif args.batched_graphs > 0:
        batched = batched_sample(lpa, torch, stream, args.batched_graphs)
    serving = None
    if args.serving_requests > 0:
        import lpa_inputs as L
        big = L.rmat(24, 16, seed=3) if args.serving_big_every > 0 else None
        serving = serving_sample(lpa, torch, stream, rate=2000.0, seconds=args.serving_requests / 2000.0,
                                 pool_size=48, big=big, big_every=args.serving_big_every if big is not None else 0)
        serving["sample"] = (f"{args.serving_requests} requests, Poisson arrivals at 2000 req/s, graphs of the "
                             "batched distribution (pool of 48)" +
                             (f"; an R-MAT scale 24 edge-factor-16 request every {args.serving_big_every}"
                              if big is not None else "; no R-MAT scale 24 request"))
        del big

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {**run_config(args, world), **({"autotuned": tuned} if tuned else {})},
                "touched_edges_per_s": touched / (ms / 1e3),
                "e2e": {"value": e2e_edges / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
                "gpu_launches": int(launches), "clocks": clocks, "roofline": roofline, "kernels": kernels,
                "cpu_baseline": cpu, "cpu_parallel": cpu_par, "per_run": per_run, "extras": extras,
                "batched": batched, "serving": serving}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
