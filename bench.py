#!/usr/bin/env python3
"""Benchmark: single-source direction-optimized BFS over a degree-separated graph
on one GB300, GTEPS as the harmonic mean over 64 seeded sources.

Workload (default): RMAT scale 26 (67,108,864 vertices, edge factor 16, a,b,c,d =
.57,.19,.19,.05, ids permuted, self-loops and duplicates removed), degree
threshold TH = 64, direction rule Beamer-stay with alpha = 10 / beta = 18, 64
seeded non-isolated sources, one query at a time through the persistent level-loop kernel.  A step is one BFS
from each of the 64 sources.  GTEPS per run = unique undirected edges of the
traversed component / device time of the run (CUDA events on the launching
stream); the reported value is their harmonic mean.  The graph build is set-up,
not timed (Graph500 convention).  Inputs are larger than L2, and the L2 is also
flushed (256 MiB write) before every timed run.

Also reported on the same line: the roofline of the level-loop kernel (the
algorithmic bytes of every run, level by level from its counters, over its
device time, against the measured HBM bandwidth), the end-to-end form with host
result buffers, the device clocks during the timed region, the CPU oracle timed
on the host as a reference, and extras: RMAT scale 22 with its TH sweep, the
Erdos-Renyi graph of 2^26 vertices / average degree 32, the batched form and the
serving loop.

`--impl reference` times the CPU oracle alone on the same workload.
Multi-GPU (torchrun): independent replicas, one graph per GPU, no data exchange.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GTEPS (harmonic mean, 64 sources) at 1 GB300"
L2_FLUSH_BYTES = 256 << 20
N_SOURCES = 64

WORKLOADS = {
    "rmat22": dict(kind="rmat", scale=22, th=64, seed=22, src_seed=2201),
    "rmat26": dict(kind="rmat", scale=26, th=64, seed=26, src_seed=2601),
    "er26": dict(kind="er", scale=26, avgdeg=32, th=64, seed=126, src_seed=12601),
    "rmat16": dict(kind="rmat", scale=16, th=64, seed=16, src_seed=1601),
    "rmat24": dict(kind="rmat", scale=24, th=64, seed=24, src_seed=2401),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---- inputs ---------------------------------------------------------------------------------

def make_edges_device(w):
    import graphgen

    if w["kind"] == "rmat":
        return graphgen.rmat_device(w["scale"], seed=w["seed"])
    n = 1 << w["scale"]
    return graphgen.er_device(n, n * w["avgdeg"] // 2, seed=w["seed"])


def make_edges_host(w):
    import graphgen

    if w["kind"] == "rmat":
        return graphgen.rmat_host(w["scale"], seed=w["seed"])
    n = 1 << w["scale"]
    return graphgen.er_host(n, n * w["avgdeg"] // 2, seed=w["seed"])


def sources_for(w, mask, rank=0):
    import graphgen

    return graphgen.sample_sources(mask, N_SOURCES, seed=w["src_seed"] + 7919 * rank)


def hmean(xs):
    xs = [x for x in xs if x > 0]
    return len(xs) / sum(1.0 / x for x in xs) if xs else 0.0


def gmean(xs):
    xs = [x for x in xs if x > 0]
    return math.exp(sum(math.log(x) for x in xs) / len(xs)) if xs else 0.0


# ---- algorithmic bytes ----------------------------------------------------------------------

def level_list(st):
    """The logged levels of a run as plain dicts (direction and counters)."""
    out = []
    for i in range(st.logged_levels):
        lv = st.level[i]
        out.append({"dir": int(lv.direction), "frontier": int(lv.frontier), "m_f": int(lv.frontier_edges),
                    "scanned": int(lv.scanned), "k": int(lv.edges_examined), "found": int(lv.found),
                    "queue": int(lv.queue_entries)})
    return out


def algorithmic_bytes(levels, n, n_ni, d):
    """Bytes one BFS must move, level by level, whatever the kernel does beyond
    them (Sec. IV-A forward visit, Sec. II-C / IV-B backward visit, Sec. VI-A.3
    output); the device computes the same count from the same counters
    (bfs_stats.model_bytes).  B = one pass over the visited bitmap (4 bytes per
    32 non-isolated vertices), D = over its delegate prefix.
      forward level:  per frontier vertex its offset pair (8 B), per row entry
                      its column and one state probe (8 B), per newly reached
                      vertex depth, parent and its queue entry written now and
                      read by the next level (16 B);
      backward level: one pass over the visited bitmap (B), per scanned vertex
                      its offset pair (8 B), per examined entry its column and
                      the frontier probe (8 B), depth, parent and the frontier
                      bit of each vertex found (12 B);
      level end:      the delegate and the whole bitmap, read and written
                      (2 (D + B)), and the next level's queue (4 B per entry)
                      when that level is forward; none after a level that found
                      nothing;
      output:         depth and parent of all n vertices (8n B), once per run.
    Returns (total, per-level bytes by phase: forward_expand,
    forward_level_end, backward_level)."""
    B = 4 * ((n_ni + 31) // 32)
    D = 4 * ((d + 31) // 32)
    ph = {"forward_expand": 0, "forward_level_end": 0, "backward_level": 0}
    for i, lv in enumerate(levels):
        end = 0
        if lv["found"] > 0:
            end = 2 * (D + B)
            if i + 1 < len(levels) and levels[i + 1]["dir"] == 0:
                end += 4 * levels[i + 1]["queue"]
        if lv["dir"] == 0:
            ph["forward_expand"] += 8 * lv["frontier"] + 8 * lv["m_f"]
            ph["forward_level_end"] += 16 * lv["found"] + end
        else:
            ph["backward_level"] += B + 8 * lv["scanned"] + 8 * lv["k"] + 12 * lv["found"] + end
    return sum(ph.values()) + 8 * n, ph


# ---- clocks during the timed region ---------------------------------------------------------

class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for_smi(torch):
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return os.environ.get("LOCAL_RANK", "0")


# ---- roofline inputs ------------------------------------------------------------------------

def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return 6800.0, "fallback"


LEVEL_LOOP_SOURCES = ("bfs_internal.cuh", "bfs_run.cu", "device_common.cuh")


def kernel_source_sha():
    """Digest of the sources that define the level-loop kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1803_03922_gb300", "csrc")
    for f in LEVEL_LOOP_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload):
    """dram bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_bfs_level_loop_%s.txt" % workload)
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha") != kernel_source_sha():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---- device runs ----------------------------------------------------------------------------

class DeviceWorkload:
    def __init__(self, name, w, rank, keep_host_edges=False, th=None, stream=None):
        import torch

        import graphgen
        import paper_1803_03922_gb300 as bfs

        self.name, self.w = name, w
        self.n = 1 << w["scale"]
        self.th = w["th"] if th is None else th
        src, dst = make_edges_device(w)
        self.m = src.numel()
        mask = graphgen.nonisolated_mask_device(self.n, src, dst).cpu().numpy()
        self.sources = sources_for(w, mask, rank)
        self.host_edges = (src.cpu().numpy(), dst.cpu().numpy()) if keep_host_edges else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.g = bfs.Graph(src, dst, self.n, th=self.th, stream=stream)
        torch.cuda.synchronize()
        self.build_s = time.perf_counter() - t0
        del src, dst
        torch.cuda.empty_cache()
        self.info = self.g.info
        self.depth = torch.empty(self.n, dtype=torch.int32, device="cuda")
        self.parent = torch.empty(self.n, dtype=torch.int32, device="cuda")
        # untimed pass: per-source traversal size, byte counts and level log
        self.ce, self.alg, self.levels, self.dirs, self.phase = [], [], [], [], []
        # per phase: [algorithmic bytes, device ns] summed over the sources (level log)
        self.phases = {"forward_expand": [0, 0], "forward_level_end": [0, 0], "backward_level": [0, 0]}
        self.setup_result_ns = 0
        for s in self.sources:
            _, _, st = self.g.run(int(s), self.depth, self.parent, stats=True)
            self.ce.append(st.component_edges)
            lvls = level_list(st)
            _, by_phase = algorithmic_bytes(lvls, self.n, self.info.n_nonisolated, self.info.delegates)
            self.alg.append(st.model_bytes)  # the same count, computed on the device side
            self.levels.append(st.levels)
            self.dirs.append("".join("B" if lv["dir"] else "T" for lv in lvls))
            td = bu = 0
            for k in by_phase:
                self.phases[k][0] += by_phase[k]
            for i in range(st.logged_levels):
                lv = st.level[i]
                dt = lv.t_end_ns - lv.t_begin_ns
                if lv.direction:
                    bu += dt
                    self.phases["backward_level"][1] += dt
                else:
                    td += dt
                    self.phases["forward_expand"][1] += lv.t_expand_ns - lv.t_begin_ns
                    self.phases["forward_level_end"][1] += lv.t_end_ns - lv.t_expand_ns
            self.setup_result_ns += st.setup_ns + st.result_ns
            self.phase.append((td, bu, st.device_ns))

    def phase_roofline(self, peak):
        """Algorithmic bytes / device time of each phase over all sources (device
        timer of the level log; each phase's time ends at the grid barrier that
        closes it), and the set-up plus result pass's share of the device time."""
        out = {}
        for k, (b, ns) in self.phases.items():
            if ns > 0:
                out[k] = {"algorithmic_gb": b / 1e9, "ms": ns / 1e6, "achieved_gbs": b / ns, "frac": b / ns / peak}
        dev = sum(p[2] for p in self.phase)
        if dev:
            out["setup_and_result_share"] = self.setup_result_ns / dev
        return out

    def timed(self, steps, flush, stream):
        """steps x len(sources) runs; returns per-run device seconds (CUDA events)."""
        import torch

        ev = []
        for _ in range(steps):
            for s in self.sources:
                if flush is not None:
                    flush.add_(1)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                self.g.run(int(s), self.depth, self.parent, stream=stream)
                b.record(stream)
                ev.append((a, b))
        torch.cuda.synchronize()
        self.g.wait(stream)
        return [a.elapsed_time(b) / 1e3 for a, b in ev]

    def gteps(self, times):
        k = len(self.sources)
        return [self.ce[i % k] / t / 1e9 for i, t in enumerate(times)]

    def close(self):
        self.g.close()


def e2e_runs(dw, steps):
    """Through the public calls with pinned host result buffers, the device->host
    copies of depth and parent inside the timed region.  A step is bfs_run_many
    over the 64 sources (run i+1 computes while run i's results cross the host
    link; results land in a ring of 4 pinned buffer pairs); the single-call form
    times one synchronous bfs_run per source."""
    import numpy as np
    import torch

    import paper_1803_03922_gb300 as bfs

    ring = 4
    hd = [torch.empty(dw.n, dtype=torch.int32).pin_memory() for _ in range(ring)]
    hp = [torch.empty(dw.n, dtype=torch.int32).pin_memory() for _ in range(ring)]
    src_host = [int(x) for x in torch.tensor(dw.sources, dtype=torch.int32).pin_memory()]
    k = len(src_host)
    status = np.zeros(k, np.int32)
    bfs.bfs_run_many(dw.g.handle, src_host[:2], hd[:2], hp[:2])  # staging buffers made outside the timing
    step_s = []
    for _ in range(steps):
        t0 = time.perf_counter()
        bfs.bfs_run_many(dw.g.handle, src_host, [hd[i % ring] for i in range(k)], [hp[i % ring] for i in range(k)],
                         status)
        step_s.append(time.perf_counter() - t0)
        if status.any():
            raise RuntimeError("bfs_run_many reported a failed run")
    pipelined = sum(dw.ce) / statistics.median(step_s) / 1e9
    ts = []
    for i in range(k):
        t0 = time.perf_counter()
        bfs.bfs_run(dw.g.handle, src_host[i], hd[0], hp[0])
        ts.append(time.perf_counter() - t0)
    single = hmean([dw.ce[i] / t / 1e9 for i, t in enumerate(ts)])
    return pipelined, single, 1e3 * statistics.median(step_s) / k, 1e3 * statistics.median(ts)


def cpu_oracle_sample(w, host_edges, sources, ce_dev, budget_s=20.0, max_sources=8):
    """The CPU oracle as it stands, single-threaded, on the same graph: a few of the
    same sources, as many as fit the time budget."""
    import oracle

    src, dst = host_edges if host_edges is not None else make_edges_host(w)
    t0 = time.perf_counter()
    og = oracle.Graph(1 << w["scale"], src, dst)
    build_s = time.perf_counter() - t0
    vals, used, spent = [], 0, 0.0
    for s in sources[:max_sources]:
        t0 = time.perf_counter()
        d, _ = og.bfs(int(s))
        dt = time.perf_counter() - t0
        ce = og.component_edges(d)
        vals.append(ce / dt / 1e9)
        used += 1
        spent += dt
        if spent > budget_s:
            break
    og.close()
    return {"value": hmean(vals), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": "%d of the %d sources on the same graph (single-threaded C, -O2; host graph build "
                      "%.1f s untimed)" % (used, len(sources), build_s),
            "seconds": spent, "host": host_cpu()}


def host_cpu():
    """The host's CPU model and logical core count (the CPU baseline runs on one)."""
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
                 "0xd49": "Arm Neoverse N2"}
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                value = line.split(":", 1)[1].strip() if ":" in line else ""
                if key == "model name" and value:
                    model = value
                    break
                if key == "cpu part" and value:
                    model = "%s (part %s)" % (arm_parts.get(value, "Arm"), value)
                    break
    except OSError:
        pass
    return {"model": model, "arch": platform.machine(), "nproc": os.cpu_count()}


# ---- main arms ------------------------------------------------------------------------------

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_value(run_s, wall_s, edges, device):
    """Replicas (one graph and one source set per rank, no data exchange): the
    whole job's GTEPS = all ranks' traversed edges / the slowest rank's device
    time.  Returns (value, max device seconds, max wall seconds)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([run_s, wall_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(edges)], dtype=torch.float64, device=device)
    dist.all_reduce(e)
    run_max, wall_max = float(t[0]), float(t[1])
    return float(e[0]) / run_max / 1e9, run_max, wall_max


class OracleInfo:
    """nnz, delegates and non-isolated vertices of the oracle's graph, the same
    description the device graph gives of itself."""

    def __init__(self, og, th):
        import numpy as np

        deg = og.degree()
        self.nnz = og.nnz
        self.delegates = int(np.count_nonzero(deg > th))
        self.n_nonisolated = int(np.count_nonzero(deg > 0))


def oracle_runs(og, sources, threads):
    """One oracle BFS per source, up to `threads` at a time (each run is the
    single-threaded oracle; runs share the read-only graph).  Returns per-run
    (seconds, GTEPS)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(s):
        t0 = time.perf_counter()
        d, _ = og.bfs(int(s))
        dt = time.perf_counter() - t0
        return dt, og.component_edges(d) / dt / 1e9

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        return list(ex.map(one, sources))


def run_reference(args, w, ws, rank):
    """CPU oracle arm: each step is one BFS of the oracle (single-threaded) from
    one of the same seeded sources on the same graph.  So that the whole run
    stays within minutes at scale 26, independent runs go on up to one host core
    each, concurrently; a run's time is its own wall time."""
    if rank != 0:
        return
    import graphgen
    import oracle

    src, dst = make_edges_host(w)
    n = 1 << w["scale"]
    mask = graphgen.nonisolated_mask_host(n, src, dst)
    sources = sources_for(w, mask, 0)
    og = oracle.Graph(n, src, dst)
    del src, dst
    info = OracleInfo(og, w["th"])
    k = len(sources)
    threads = min(os.cpu_count() or 1, 16, max(1, args.steps))
    oracle_runs(og, [sources[i % k] for i in range(args.warmup)], threads)
    res = oracle_runs(og, [sources[(args.warmup + i) % k] for i in range(args.steps)], threads)
    ts = [r[0] for r in res]
    v = hmean([r[1] for r in res])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded RMAT, Graph500 parameters)",
        "config": dict(config_of(args.workload, w, info), parallelism="replicas" if ws > 1 else "single GPU"),
        "cpu_baseline": {"kind": "oracle", "cores": threads, "value": v, "unit": "GTEPS",
                         "sample": "one of the 64 seeded sources per step on the same graph; each run is the "
                                   "single-threaded C oracle (-O2), up to %d runs at a time on separate host "
                                   "cores" % threads, "host": host_cpu()},
        "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    og.close()
    print(json.dumps(line), flush=True)


# ---- batched form and serving loop ----------------------------------------------------------

SERVE_GRAPHS = [
    ("rmat18", dict(kind="rmat", scale=18, th=64, seed=18, src_seed=1801)),
    ("rmat20", dict(kind="rmat", scale=20, th=64, seed=20, src_seed=2001)),
    ("rmat22", dict(kind="rmat", scale=22, th=64, seed=22, src_seed=2201)),
    ("rmat24", dict(kind="rmat", scale=24, th=64, seed=24, src_seed=2401)),
    ("er22", dict(kind="er", scale=22, avgdeg=16, th=64, seed=122, src_seed=12201)),
]
SERVE_RATES = (1000, 4000, 16000)
SERVE_SOURCES = 1024
SERVE_POOL = 160  # output buffer pairs per graph (queries outstanding before the client waits)


def build_served_graph(w):
    import torch

    import graphgen
    import paper_1803_03922_gb300 as bfs

    n = 1 << w["scale"]
    src, dst = make_edges_device(w)
    mask = graphgen.nonisolated_mask_device(n, src, dst).cpu().numpy()
    sources = graphgen.sample_sources(mask, SERVE_SOURCES, seed=w["src_seed"])
    g = bfs.Graph(src, dst, n, th=w["th"])
    del src, dst
    torch.cuda.empty_cache()
    return g, sources


def batched_vs_single(g, sources, batches=8):
    """64-lane batches against one query at a time on the same graph and sources:
    queries/s from CUDA events over `batches` x 64 queries, parents included, and
    the aggregate GTEPS (the queries' traversed component edges / time)."""
    import numpy as np
    import torch

    import paper_1803_03922_gb300 as bfs

    n = g.n
    out = {}
    edges = None  # traversed component edges of the timed batches' queries (untimed stats runs)
    for with_par in (True, False):
        b = bfs.Batch(g, with_parents=with_par)
        depth = torch.empty((64, n), dtype=torch.uint8, device="cuda")
        parent = torch.empty((64, n), dtype=torch.int32, device="cuda") if with_par else None
        if edges is None:
            edges = 0
            for i in range(batches):
                _, _, st = b.run(sources[64 * i:64 * (i + 1)], depth, parent, stats=True)
                edges += st.traversed_edges
        for i in range(2):
            b.run(sources[64 * i:64 * (i + 1)], depth, parent)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(batches):
            b.run(sources[64 * i:64 * (i + 1)], depth, parent)
        e1.record()
        torch.cuda.synchronize()
        b.wait()
        ms = e0.elapsed_time(e1)
        out["batched_qps" if with_par else "batched_depth_only_qps"] = 64 * batches / ms * 1e3
        out["ms_per_batch" if with_par else "ms_per_batch_depth_only"] = ms / batches
        out["gteps_aggregate" if with_par else "gteps_aggregate_depth_only"] = edges / (ms / 1e3) / 1e9
        b.close()
        del depth, parent
        torch.cuda.empty_cache()
    d1 = torch.empty(n, dtype=torch.int32, device="cuda")
    p1 = torch.empty(n, dtype=torch.int32, device="cuda")
    for s in sources[:4]:
        g.run(int(s), d1, p1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for s in sources[:64 * batches]:
        g.run(int(s), d1, p1)
    e1.record()
    torch.cuda.synchronize()
    g.wait()
    ms = e0.elapsed_time(e1)
    out["single_qps"] = 64 * batches / ms * 1e3
    out["single_gteps_aggregate"] = edges / (ms / 1e3) / 1e9
    out["speedup"] = out["batched_qps"] / out["single_qps"]
    # the same queries grouped for batching (bfs_batch_order: by the degree sum of
    # each source's neighbours), parents included
    qs = np.asarray(sources[:64 * batches], dtype=np.int32)
    grouped = qs[bfs.bfs_batch_order(g.handle, qs)]
    b = bfs.Batch(g, with_parents=True)
    depth = torch.empty((64, n), dtype=torch.uint8, device="cuda")
    parent = torch.empty((64, n), dtype=torch.int32, device="cuda")
    for i in range(2):
        b.run(grouped[64 * i:64 * (i + 1)], depth, parent)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(batches):
        b.run(grouped[64 * i:64 * (i + 1)], depth, parent)
    e1.record()
    torch.cuda.synchronize()
    b.wait()
    ms = e0.elapsed_time(e1)
    out["batched_grouped_qps"] = 64 * batches / ms * 1e3
    out["gteps_aggregate_grouped"] = edges / (ms / 1e3) / 1e9
    out["speedup_grouped"] = out["batched_grouped_qps"] / out["single_qps"]
    b.close()
    del depth, parent
    torch.cuda.empty_cache()
    # the batched schedule autotuned (Beamer alpha of the union frontier), then timed as above
    from paper_1803_03922_gb300.autotune import tune_batch_alpha

    alpha0 = g.opt.alpha
    best, cand = tune_batch_alpha(g, sources, batches=2)
    b = bfs.Batch(g, with_parents=True)
    depth = torch.empty((64, n), dtype=torch.uint8, device="cuda")
    parent = torch.empty((64, n), dtype=torch.int32, device="cuda")
    b.run(sources[:64], depth, parent)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(batches):
        b.run(sources[64 * i:64 * (i + 1)], depth, parent)
    e1.record()
    torch.cuda.synchronize()
    b.wait()
    ms = e0.elapsed_time(e1)
    out["autotuned_alpha"] = best
    out["autotuned_batched_qps"] = 64 * batches / ms * 1e3
    out["autotuned_candidates_ms_per_batch"] = {str(a): round(t * 1e3, 3) for a, t in cand.items()}
    b.close()
    g.set_options(alpha=alpha0)
    return out


def serve_trace(rate, count, n_graphs, n_sources, seed):
    """Open-loop Poisson arrivals: (offset ns, graph id, source index), graphs uniform."""
    import numpy as np

    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1e9 / rate, count)
    offs = np.cumsum(gaps).astype(np.int64)
    gids = rng.integers(0, n_graphs, count)
    idx = rng.integers(0, n_sources, count)
    return list(zip(offs.tolist(), gids.tolist(), idx.tolist()))


def latency_summary(lat_ns, t_first, t_last, count):
    import numpy as np

    lat = np.asarray(lat_ns, dtype=np.float64) / 1e6
    span = (t_last - t_first) / 1e9
    return {"queries": count, "qps": count / span if span > 0 else None,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean())}


def serve_open_loop(srv, graphs, sources, pools, trace):
    """Submits each query at its arrival time (through bfs_server_submit with that
    arrival stamp) and collects completions; returns the latency summary."""
    import paper_1803_03922_gb300 as bfs

    h = srv._h
    t0 = bfs.bfs_server_now_ns() + 2_000_000
    i, outstanding, lat, bad = 0, {}, [], 0
    t_last = t0
    while i < len(trace) or outstanding:
        now = bfs.bfs_server_now_ns()
        while i < len(trace) and t0 + trace[i][0] <= now:
            off, gid, si = trace[i]
            if not pools[gid]:
                break  # the client has no free result buffer for this graph: wait
            d, p = pools[gid].pop()
            t = bfs.bfs_server_submit(h, gid, int(sources[gid][si]), d, p, t0 + off)
            outstanding[t] = (gid, d, p)
            i += 1
        for rec in bfs.bfs_server_poll(h, 256, 0 if i < len(trace) else 5):
            gid, d, p = outstanding.pop(rec.ticket)
            pools[gid].append((d, p))
            lat.append(rec.t_done_ns - rec.t_arrival_ns)
            bad += rec.status != 0
            t_last = max(t_last, rec.t_done_ns)
    out = latency_summary(lat, t0, t_last, len(trace))
    out["failed"] = bad
    return out


def one_at_a_time(graphs, sources, trace, stream):
    """The same arrivals served FIFO, one bfs_run (single-source kernel, whole
    device) per query, each checked for its device status before the next."""
    import torch

    import paper_1803_03922_gb300 as bfs

    outs = [(torch.empty(g.n, dtype=torch.int32, device="cuda"),
             torch.empty(g.n, dtype=torch.int32, device="cuda")) for g in graphs]
    t0 = bfs.bfs_server_now_ns() + 2_000_000
    lat = []
    for off, gid, si in trace:
        ta = t0 + off
        while bfs.bfs_server_now_ns() < ta:
            pass
        g = graphs[gid]
        g.run(int(sources[gid][si]), outs[gid][0], outs[gid][1], stream=stream)
        g.wait(stream)
        lat.append(bfs.bfs_server_now_ns() - ta)
    t_last = t0 + trace[-1][0] + lat[-1]
    return latency_summary(lat, t0, t_last, len(trace))


def serving_bench(stream, rates=SERVE_RATES, duration_s=1.5, single_cap=2000, max_concurrent=2):
    """Serving loop over five device-resident graphs (RMAT scales 18/20/22/24 and
    Erdos-Renyi 2^22 with average degree 16): Poisson arrivals at each rate, uniform
    over graphs and over each graph's non-isolated sources; the server against the
    same arrivals served one at a time.  Also a saturation run (every query
    arrives at once): the server's peak queries/s, with its default grouped
    batches and with batches in arrival order."""
    import torch

    import paper_1803_03922_gb300 as bfs

    graphs, sources = [], []
    for name, w in SERVE_GRAPHS:
        g, s = build_served_graph(w)
        graphs.append(g)
        sources.append(s)
    srv = bfs.Server(max_concurrent=max_concurrent, max_lanes=64, with_parents=True)
    for g in graphs:
        srv.add_graph(g)
    pools = [[(torch.empty(g.n, dtype=torch.uint8, device="cuda"), torch.empty(g.n, dtype=torch.int32, device="cuda"))
              for _ in range(SERVE_POOL)] for g in graphs]
    out = {"graphs": [name for name, _ in SERVE_GRAPHS], "max_concurrent": max_concurrent,
           "pool_per_graph": SERVE_POOL, "one_at_a_time_queries": single_cap, "rates": {}}
    # warm-up: every graph's contexts
    serve_open_loop(srv, graphs, sources, pools, serve_trace(20000, 400, len(graphs), SERVE_SOURCES, 1))
    for rate in rates:
        trace = serve_trace(rate, max(200, int(rate * duration_s)), len(graphs), SERVE_SOURCES, rate)
        r = {"server": serve_open_loop(srv, graphs, sources, pools, trace)}
        r["one_at_a_time"] = one_at_a_time(graphs, sources, trace[:single_cap], stream)
        out["rates"][str(rate)] = r
    sat = serve_trace(1e9, 4000, len(graphs), SERVE_SOURCES, 99)
    out["saturation_server"] = serve_open_loop(srv, graphs, sources, pools, sat)
    out["saturation_one_at_a_time"] = one_at_a_time(graphs, sources, sat[:single_cap], stream)
    out["server_stats"] = srv.stats()
    srv.close()
    # the same saturation run with batches taken in arrival order (group_batches off)
    fifo = bfs.Server(max_concurrent=max_concurrent, max_lanes=64, with_parents=True, group_batches=False)
    for g in graphs:
        fifo.add_graph(g)
    serve_open_loop(fifo, graphs, sources, pools, serve_trace(20000, 400, len(graphs), SERVE_SOURCES, 1))
    out["saturation_server_arrival_order"] = serve_open_loop(fifo, graphs, sources, pools, sat)
    fifo.close()
    del pools
    for g in graphs:
        g.close()
    torch.cuda.empty_cache()
    return out


def autotuned(w, rank, flush, stream, peak):
    """The autotuner (TH, alpha/beta, CTAs per SM, direction rule, per-level mask)
    tuned on 16 of the 64 sources, then the tuned graph timed on all 64 like the
    benchmark value."""
    import torch

    from paper_1803_03922_gb300.autotune import device_tuner, th_space_for_scale

    src, dst = make_edges_device(w)
    n = 1 << w["scale"]
    import graphgen

    mask = graphgen.nonisolated_mask_device(n, src, dst).cpu().numpy()
    sources = sources_for(w, mask, rank)
    t0 = time.perf_counter()
    res, g = device_tuner(src, dst, n, [int(x) for x in sources[:16]], runs=2, ths=th_space_for_scale(w["scale"]))
    tune_s = time.perf_counter() - t0
    del src, dst
    torch.cuda.empty_cache()
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    ce = []
    for s in sources:
        _, _, st = g.run(int(s), depth, parent, stats=True)
        ce.append(st.component_edges)
    ts = []
    for rep in range(2):
        for s in sources:
            flush.add_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.run(int(s), depth, parent, stream=stream)
            b.record(stream)
            ts.append((a, b))
    torch.cuda.synchronize()
    g.wait(stream)
    times = [a.elapsed_time(b) / 1e3 for a, b in ts][len(sources):]
    g.close()
    opts = {k: (v if not isinstance(v, float) else round(v, 4)) for k, v in res.options.items()}
    return {"gteps": hmean([ce[i] / t / 1e9 for i, t in enumerate(times)]), "th": res.th, "options": opts,
            "tuning_speedup_on_sample": res.speedup, "trials": len(res.trials), "tune_s": tune_s}


DEGREE_THS = (2, 4, 8, 16, 32, 64, 128, 256, 512, 1024)


def degree_table(rows):
    """Compact rows of Graph.degree_classes: TH, delegate % of vertices, nn/nd/dd % of entries."""
    return [[r["th"], round(r["delegate_pct"], 4), round(r["nn_pct"], 3), round(r["nd_pct"], 3),
             round(r["dd_pct"], 3)] for r in rows]


def serving_extras(stream):
    out = {}
    try:
        g, srcs = build_served_graph(WORKLOADS["rmat24"])
        out["batched_rmat24"] = batched_vs_single(g, srcs)
        g.close()
    except Exception as e:  # report, do not hide
        out["batched_rmat24"] = {"error": str(e)}
    try:
        out["serving"] = serving_bench(stream)
    except Exception as e:
        out["serving"] = {"error": str(e)}
    return out


def config_of(name, w, info=None):
    c = {"workload": name, "graph": "RMAT" if w["kind"] == "rmat" else "Erdos-Renyi", "scale": w["scale"],
         "n": 1 << w["scale"], "th": w["th"], "schedule": "beamer_stay", "alpha": 10, "beta": 18,
         "sources": N_SOURCES,
         "graph_seed": w["seed"], "source_seed": w["src_seed"],
         "l2": "inputs larger than L2 and L2 flushed (256 MiB write) before every timed run"}
    if w["kind"] == "rmat":
        c.update(edge_factor=16, abcd=[0.57, 0.19, 0.19, 0.05])
    else:
        c.update(avg_degree=w["avgdeg"])
    if info is not None:
        c.update(nnz=info.nnz, delegates=info.delegates, nonisolated=info.n_nonisolated,
                 adjacency_bytes=info.nnz * 4 + (info.n_nonisolated + 1) * 8)
    return c


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat26", choices=sorted(WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip the TH sweep and the scale-26 graphs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--serving-only", action="store_true", help="print only the batched and serving measurements")
    ap.add_argument("--batched-only", metavar="GRAPH", choices=sorted(WORKLOADS),
                    help="print only the 64-lane batched measurement on GRAPH")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w, ws, rank)
        return

    import torch

    torch.cuda.set_device(local)
    if args.serving_only:
        print(json.dumps(serving_extras(torch.cuda.current_stream())), flush=True)
        return
    if args.batched_only:
        g, srcs = build_served_graph(WORKLOADS[args.batched_only])
        print(json.dumps({args.batched_only: batched_vs_single(g, srcs)}), flush=True)
        g.close()
        return
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    dw = DeviceWorkload(args.workload, w, rank, keep_host_edges=(rank == 0 and ws == 1 and not args.no_cpu))
    log("[bench] %s: n=%d nnz=%d d=%d build %.2fs, levels %s" % (
        args.workload, dw.n, dw.info.nnz, dw.info.delegates, dw.build_s, sorted(set(dw.levels))))
    dw.timed(args.warmup, flush, stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    sampler = ClockSampler(gpu_id_for_smi(torch))
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    times = dw.timed(args.steps, flush, stream)
    t_all1.record(stream)
    barrier()
    clocks = sampler.stop()
    wall = t_all0.elapsed_time(t_all1) / 1e3
    run_s = sum(times)
    if ws > 1:
        value, run_max, wall = replica_value(run_s, wall, float(sum(dw.ce) * args.steps), "cuda")
    else:
        value = hmean(dw.gteps(times))
        run_max = run_s
    k = len(dw.sources)
    alg_total = sum(dw.alg[i % k] for i in range(len(times)))
    achieved = alg_total / run_s / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = ncu_traffic(args.workload)
    e2e_val, e2e_single, e2e_ms_pipelined, e2e_ms_single = e2e_runs(dw, max(1, min(args.steps, 3)))
    td_ns = sum(p[0] for p in dw.phase)
    bu_ns = sum(p[1] for p in dw.phase)
    dev_ns = sum(p[2] for p in dw.phase)
    paper_style = gmean([(16 << w["scale"]) / t / 1e9 for i, t in enumerate(times) if dw.levels[i % k] > 2])
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * run_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded RMAT, Graph500 parameters)",
        "config": dict(config_of(args.workload, w, dw.info),
                       parallelism="replicas" if ws > 1 else "single GPU"),
        "gpu_launches": 2 * len(times),  # per BFS: the level loop and the result pass
        "clocks": clocks,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "bfs_level_loop", "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_total / len(times),
                     "traffic_over_algorithmic": traffic / (alg_total / len(times)) if traffic else None,
                     "launch_ms_mean": 1e3 * run_s / len(times)},
        "e2e": {"value": e2e_val, "unit": "GTEPS", "h2d_bytes_per_step": 4 * k,
                "d2h_bytes_per_step": 8 * dw.n * k},
        "detail": {"wall_ms_per_step_with_flush": 1e3 * wall / args.steps,
                   "gteps_aggregate": sum(dw.ce[i % k] for i in range(len(times))) / run_s / 1e9,
                   "gteps_paper_style_geomean": paper_style,
                   "ms_per_bfs_median": 1e3 * statistics.median(times),
                   "build_s": dw.build_s, "levels": statistics.median(dw.levels),
                   "directions_first_source": dw.dirs[0],
                   "forward_share": td_ns / dev_ns if dev_ns else None,
                   "backward_share": bu_ns / dev_ns if dev_ns else None,
                   "phase_roofline": dw.phase_roofline(peak),
                   "e2e_ms_per_bfs_pipelined": e2e_ms_pipelined,
                   "e2e_single_call_gteps": e2e_single,
                   "e2e_single_call_ms_per_bfs_median": e2e_ms_single},
    }
    if rank == 0 and not args.no_extras:
        # the same graph and sources under plain Beamer alpha 15 / beta 18 (the
        # direction rule before this build's default), for comparison
        dw.g.set_options(schedule=0, alpha=15)
        dw.timed(1, flush, stream)
        tb = dw.timed(1, flush, stream)
        line["detail"]["plain_beamer_a15"] = {"gteps": hmean(dw.gteps(tb)),
                                              "ms_per_bfs_mean": 1e3 * statistics.mean(tb)}
        dw.g.set_options(schedule=7, alpha=10)
    host_edges = dw.host_edges
    sources = dw.sources
    ce_dev = dw.ce
    degree_rows = dw.g.degree_classes(DEGREE_THS)
    dw.close()
    del dw

    if rank == 0 and not args.no_extras:
        from paper_1803_03922_gb300.autotune import th_for_scale, th_space_for_scale

        extras = {"degree_classes_%s" % args.workload: degree_table(degree_rows),
                  "th_rule": {"rule": "64 * 2^((scale - 30) / 2) (Sec. VI-B)",
                              "th_by_scale": {str(sc): th_for_scale(sc) for sc in (16, 22, 24, 26, 30, 32)}}}
        w22 = WORKLOADS["rmat22"]
        for th in [w22["th"]] + [t for t in th_space_for_scale(22) if t != w22["th"]]:
            if args.workload == "rmat22" and th == w22["th"]:
                continue
            try:
                d2 = DeviceWorkload("rmat22", w22, rank, th=th)
                d2.timed(1, flush, stream)
                t2 = d2.timed(2, flush, stream)
                key = "rmat22" if th == w22["th"] else "rmat22_th%d" % th
                extras[key] = {"gteps": hmean(d2.gteps(t2)), "delegates": d2.info.delegates,
                               "ms_per_bfs_median": 1e3 * statistics.median(t2),
                               "roofline_frac": sum(d2.alg[i % len(d2.sources)] for i in range(len(t2)))
                               / sum(t2) / 1e9 / peak}
                if th == w22["th"]:
                    extras[key]["phase_roofline"] = d2.phase_roofline(peak)
                    extras[key]["directions_first_source"] = d2.dirs[0]
                d2.close()
            except Exception as e:  # report, do not hide
                extras["rmat22_th%d" % th] = {"error": str(e)}
        try:  # config 1: RMAT scale 16, top-down only, 64 sources
            w16 = dict(WORKLOADS["rmat16"])
            d1 = DeviceWorkload("rmat16", w16, rank)
            d1.g.set_options(schedule=1)
            d1.timed(1, flush, stream)
            t1 = d1.timed(2, flush, stream)
            extras["rmat16_topdown"] = {"gteps": hmean(d1.gteps(t1)),
                                        "ms_per_bfs_median": 1e3 * statistics.median(t1),
                                        "roofline_frac": sum(d1.alg[i % len(d1.sources)] for i in range(len(t1)))
                                        / sum(t1) / 1e9 / peak,
                                        "phase_roofline": d1.phase_roofline(peak)}
            d1.close()
        except Exception as e:  # report, do not hide
            extras["rmat16_topdown"] = {"error": str(e)}
        try:
            extras["autotuned_rmat22"] = autotuned(w22, rank, flush, stream, peak)
        except Exception as e:  # report, do not hide
            extras["autotuned_rmat22"] = {"error": str(e)}
        for key, name, th26 in (("rmat26", "rmat26", None), ("er26", "er26", None),
                                ("rmat26_th%d" % th_for_scale(26), "rmat26", th_for_scale(26))):
            if key == args.workload:
                continue
            try:
                d3 = DeviceWorkload(name, WORKLOADS[name], rank, th=th26)
                d3.timed(1, None, stream)
                t3 = d3.timed(2, None, stream)
                extras[key] = {"gteps": hmean(d3.gteps(t3)), "ms_per_bfs_median": 1e3 * statistics.median(t3),
                                "roofline_frac": sum(d3.alg[i % len(d3.sources)] for i in range(len(t3)))
                                / sum(t3) / 1e9 / peak,
                                "nnz": d3.info.nnz, "delegates": d3.info.delegates,
                                "levels": statistics.median(d3.levels), "build_s": d3.build_s,
                                "directions_first_source": d3.dirs[0],
                                "phase_roofline": d3.phase_roofline(peak)}
                d3.close()
                del d3
                torch.cuda.empty_cache()
            except Exception as e:  # report, do not hide
                extras[key] = {"error": str(e)}
        if not args.no_serving:
            extras.update(serving_extras(stream))
        line["extras"] = extras

    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample(w, host_edges, sources, ce_dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
