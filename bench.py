#!/usr/bin/env python3
"""GTEPS of single-source EIC queries on one GB300 (and N independent replicas).

Workload (default): RMAT/Kronecker scale 25, edge factor 16, a,b,c,d =
0.57,0.19,0.19,0.05, vertex ids permuted, integer weights uniform in [1, 255],
symmetrised and deduplicated on the device; 64 sources drawn uniformly from
the non-isolated vertices. A step is one pass of the whole query path
(Algorithm 1 with Function 1/2, exact distances) for the 64 sources on the
resident graph. The graph build (preprocessing, Section 4.1) is timed
separately and reported as build_s.

  value    = sum over queries of m_c (undirected edges in the source's
             component, Graph500 convention) / device time of the step, summed
             over ranks (replicas) with the max step time over ranks.
  e2e      = the same metric with every step's sources copied from pinned host
             memory and every query's distance array copied back to pinned host
             memory inside the timed region.
  roofline = algorithmic bytes of the query kernel per launch (frontier items
             16 B, traversed entries 12 B, successful relaxations 8 B, pulled
             vertices 12 B, plus 4n for dist) over the CUDA-event duration of
             one query, against the measured HBM copy bandwidth.

--impl reference runs the CPU oracle (binary-heap Dijkstra) on the host cores
for a bounded sample of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS single-source & batched vs plain path on 1 GB300; p50/p99 query latency"


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=25, help="Kronecker scale of the workload")
    ap.add_argument("--road", type=int, default=0, metavar="SIDE",
                    help="time a SIDE^2 road-like grid (weights [1,4095]) instead of the Kronecker workload "
                         "(for profiling the fused-round kernel)")
    ap.add_argument("--sources", type=int, default=64)
    ap.add_argument("--cpu-sample", type=int, default=1, help="oracle queries timed for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched measurements")
    ap.add_argument("--no-served", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-stress", action="store_true", help="skip the road-like and log-normal-weight workloads")
    ap.add_argument("--stress-sources", type=int, default=16, help="sources per stress workload")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# DRAM bytes (read + write) of one query-kernel launch on the default workload,
# from an ncu capture of dram__bytes_read.sum + dram__bytes_write.sum, valid only
# for the kernel code it was taken on: the key hashes the kernel sources without
# their comments and blank lines, and any change to the code reports null.
KERNEL_SOURCES = ("paper_2506_19349_gb300/csrc/sssp.cu", "paper_2506_19349_gb300/csrc/common.cuh",
                  "paper_2506_19349_gb300/csrc/graph.h", "paper_2506_19349_gb300/csrc/graph.cu",
                  "paper_2506_19349_gb300/csrc/stats.cuh", "include/eic.h")
MEASURED_TRAFFIC = {  # {(scale, kernel code sha256): bytes per launch}
    (25, "298c3629a5385ee6ab3745012138720b3479de107e64f161049f176bd47c3fcd"): 6088278784,
}


def strip_c_comments(text):
    """C/C++ source without // and /* */ comments (string and character
    literals kept), trailing blanks and empty lines."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (line.rstrip() for line in "".join(out).split("\n"))
    return "\n".join(line for line in lines if line)


def kernel_sources_sha256():
    import hashlib

    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(strip_c_comments(f.read()).encode())
    return h.hexdigest()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def make_workload(scale: int, nsources: int, rank: int = 0, road: int = 0):
    """The resident graph (the same on every rank) and this rank's sources
    (replicas draw their own, so N ranks process N x nsources queries)."""
    from paper_2506_19349_gb300 import graphgen

    if road:
        wl = graphgen.road(road, seed=3, wmax=4095, nsources=nsources)
        if rank:
            wl.sources = graphgen.pick_sources(wl.n, wl.src, wl.dst, nsources, 3 + 1000 * rank, "largest")
        return wl
    return graphgen.kron(scale, seed=2, nsources=nsources, source_seed=2 + 1000 * rank)


def max_over_ranks(x: float, world: int, device) -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device) -> float:
    """Sum over the ranks (units every rank processed)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_gteps(edges_all_ranks_per_step: float, steps: int, max_ms: float) -> float:
    """Edges of all ranks' queries over the slowest rank's time, in GTEPS."""
    return edges_all_ranks_per_step * steps / (max_ms * 1e-3) / 1e9


def workload_config(wl, scale, nsources, road=0):
    desc = (f"road{road}: {road}^2 grid, 4-neighbour, 10% of edges deleted, 2% diagonal shortcuts, weights uniform "
            f"[1,4095], {nsources} sources from the largest component" if road else
            f"kron{scale}: RMAT(0.57,0.19,0.19,0.05) scale {scale} edgefactor 16, ids permuted, "
            f"weights uniform [1,255], {nsources} sources uniform over non-isolated vertices")
    return {"workload": desc,
            "n": int(wl.n), "tuples": int(wl.num_tuples), "queries_per_step": nsources,
            "l2": "inputs larger than L2 (CSR of the resident graph)", "path": "plain single-source, one "
                                                                          "persistent launch per query"}


def oracle_baseline(wl, sample: int, m_c_of):
    """Time the oracle's Dijkstra (one host thread) on `sample` sources."""
    import oracle

    og = oracle.Graph(wl.n, wl.src, wl.dst, wl.w)
    total_edges, total_t = 0, 0.0
    for s in wl.sources[:sample]:
        t0 = time.perf_counter()
        d, rc = og.dijkstra(int(s))
        total_t += time.perf_counter() - t0
        total_edges += m_c_of(og, d)
    return og, total_edges / total_t / 1e9, total_t


def oracle_m_c(og, d):
    import numpy as np

    deg = og.degrees()
    return int(deg[d != 0xFFFFFFFF].sum() // 2)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.scale, args.sources, road=args.road)
    import oracle

    og = oracle.Graph(wl.n, wl.src, wl.dst, wl.w)
    srcs = [int(s) for s in wl.sources]
    times, edges = [], []
    for k in range(args.warmup + args.steps):
        s = srcs[k % len(srcs)]
        t0 = time.perf_counter()
        d, rc = og.dijkstra(s)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            edges.append(oracle_m_c(og, d))
    value = sum(edges) / sum(times) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": workload_config(wl, args.scale, args.sources, args.road),
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"one binary-heap Dijkstra query per step on kron{args.scale} (CPU "
                                       f"oracle), sources cycling through the workload's list"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _degrees(eic, g, torch):
    import numpy as np

    rowp = np.empty(g.n + 1, dtype=np.uint64)
    eic.load_library().eic_graph_export(g.handle, rowp.ctypes.data, None, None, None)
    return torch.from_numpy(np.diff(rowp).astype(np.int64)).cuda()


def _m_c(deg, d):
    return int(deg[d != -1].sum().item() // 2)


def batch_run_timed(b, stream, torch, runs):
    """Device time (ms) of each of `runs` whole-batch runs of a prepared batch."""
    out = []
    for _ in range(runs):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(stream)
        e1.record(stream)
        st = b.wait(stream)
        if (st != 0).any():
            raise RuntimeError(f"batch statuses {sorted(set(st.tolist()))}")
        out.append(e0.elapsed_time(e1))
    return out


def batched_same_workload(eic, torch, g, srcs, dists, stream, runs, plain_gteps, edges):
    """The same queries as one tuned persistent batch (eic_batch_*)."""
    import numpy as np

    ref = [eic.to_host_u32(d).copy() for d in dists]
    b = eic.Batch([g] * len(srcs), srcs, dists)
    t0 = time.perf_counter()
    cfg = b.tune(stream)
    tune_s = time.perf_counter() - t0
    batch_run_timed(b, stream, torch, 1)  # first run captures the CUDA graph
    ms = batch_run_timed(b, stream, torch, runs)
    same = all(np.array_equal(eic.to_host_u32(d), r) for d, r in zip(dists, ref))
    info = b.info()
    b.close()
    gteps = edges / (statistics.mean(ms) * 1e-3) / 1e9
    return {"value": gteps, "unit": "GTEPS", "ms_per_batch": statistics.mean(ms), "runs": runs,
            "speedup_vs_plain": gteps / plain_gteps, "identical_to_plain": same, "tune_s": tune_s,
            "config": {k: info[k] for k in ("groups", "blocks_per_group", "block_threads", "cuda_graph", "gap_shift",
                                            "heavy_min", "scratch_bytes")},
            "gpu_launches_per_batch": 2}


def batched_mixed(eic, torch, stream, runs):
    """32 graphs of uneven size x 8 sources: one tuned persistent batch vs 256
    sequential plain calls (the plain path's per-query latency is reported too)."""
    import numpy as np
    from paper_2506_19349_gb300 import graphgen

    t0 = time.perf_counter()
    wls = graphgen.batch_set()
    gen_s = time.perf_counter() - t0
    graphs, srcs, degs = [], [], []
    for wl in wls:
        g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
        deg = _degrees(eic, g, torch)
        for s in wl.sources:
            graphs.append(g)
            srcs.append(int(s))
            degs.append(deg)
    del wls
    dists = [eic.new_dist(g.n) for g in graphs]

    def plain_pass(params=None):
        evs = []
        for i, (g, s, d) in enumerate(zip(graphs, srcs, dists)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            eic.sssp(g, s, dist=d, params=params[i] if params else None)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    plain_pass()  # warm-up
    edges = sum(_m_c(deg, d) for deg, d in zip(degs, dists))
    ref = [eic.to_host_u32(d).copy() for d in dists]
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    lat = plain_pass()
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    b = eic.Batch(graphs, srcs, dists)
    t0 = time.perf_counter()
    cfg = b.tune(stream)
    tune_s = time.perf_counter() - t0
    shifts = b.gap_shifts()
    batch_run_timed(b, stream, torch, 1)  # first run captures the CUDA graph
    ms = batch_run_timed(b, stream, torch, runs)
    same = all(np.array_equal(eic.to_host_u32(d), r) for d, r in zip(dists, ref))
    info = b.info()
    b.close()
    # like for like: the plain path at the step width the tuner chose for each graph
    tuned_params = [eic.default_params(gap_shift=sh) for sh in shifts]
    plain_pass(tuned_params)  # warm-up
    p0.record(stream)
    lat_t = plain_pass(tuned_params)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_t_ms = p0.elapsed_time(p1)
    same_t = all(np.array_equal(eic.to_host_u32(d), r) for d, r in zip(dists, ref))
    lat.sort()
    lat_t.sort()
    plain_gteps = edges / (plain_ms * 1e-3) / 1e9
    plain_t_gteps = edges / (plain_t_ms * 1e-3) / 1e9
    gteps = edges / (statistics.mean(ms) * 1e-3) / 1e9
    pct = lambda v, q: v[min(len(v) - 1, int(q * len(v)))]
    return {"workload": "32 graphs: RMAT scales 12..22 (two seeds each) and grids 256^2 x3, 512^2 x3, 1024^2 x2, "
                        "2048^2 x2 (10% edges deleted, 2% diagonals), weights uniform [1,255], 8 sources each",
            "queries": len(srcs), "generate_s": gen_s,
            "plain": {"value": plain_gteps, "unit": "GTEPS", "ms": plain_ms, "gap_shift": 0,
                      "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99)}},
            "plain_tuned": {"value": plain_t_gteps, "unit": "GTEPS", "ms": plain_t_ms,
                            "gap_shift": "per graph, the batch tuner's choice", "identical_to_plain": same_t,
                            "latency_ms": {"p50": pct(lat_t, 0.5), "p99": pct(lat_t, 0.99)}},
            "batched": {"value": gteps, "unit": "GTEPS", "ms_per_batch": statistics.mean(ms), "runs": runs,
                        "tune_s": tune_s, "identical_to_plain": same, "gap_shifts": sorted(set(shifts)),
                        "config": {k: info[k] for k in ("groups", "blocks_per_group", "block_threads", "cuda_graph",
                                                        "gap_shift", "heavy_min", "scratch_bytes")}},
            "speedup": gteps / plain_t_gteps, "speedup_basis": "batched vs the plain path at the same per-graph "
                                                               "step width (like for like)",
            "speedup_vs_plain_default": gteps / plain_gteps}


def stress(eic, torch, stream, nsources):
    """The stress workloads, on the plain path: the 4096^2 road-like grid
    (weights [1,4095]) with the default step width (fused rounds, and for
    comparison without them) and with the exact 16x scaling the autotuners
    pick for grids, and Kron 25 with log-normal weights. GTEPS = edges in the
    source's component / query time."""
    import numpy as np
    from paper_2506_19349_gb300 import graphgen

    cases = (
        ("road_4096", "4096^2 grid, 4-neighbour, 10% of edges deleted, 2% diagonal shortcuts, weights uniform "
         "[1,4095], sources from the largest component",
         lambda: graphgen.road(4096, seed=3, wmax=4095, nsources=nsources),
         (("gap_shift_0", {}), ("gap_shift_0_no_fuse", {"flags": eic.FLAG_NO_FUSE}), ("gap_shift_4", {"gap_shift": 4}))),
        ("kron25_lognormal", "kron25 topology, weights clamp(llround(exp(3 + 1.5 Z)), 1, 65535), sources uniform "
         "over non-isolated vertices", lambda: graphgen.kron(25, seed=2, weights="lognormal", nsources=nsources),
         (("gap_shift_0", {}),)),
    )
    out = {}
    for name, desc, make, shifts in cases:
        t0 = time.perf_counter()
        wl = make()
        gen_s = time.perf_counter() - t0
        g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
        srcs = [int(s) for s in wl.sources]
        del wl
        deg = _degrees(eic, g, torch)
        d = eic.new_dist(g.n)
        res = {"workload": desc, "n": g.n, "m": g.m, "sources": len(srcs), "generate_s": gen_s}
        for label, kw in shifts:
            p = eic.default_params(**kw)
            eic.sssp(g, srcs[0], dist=d, params=p)  # warm-up
            ms, mc, steps, rounds = [], [], [], []
            for s in srcs:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, _, info = eic.sssp(g, s, dist=d, params=p, stats=True)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                mc.append(_m_c(deg, d))
                steps.append(info["steps"])
                rounds.append(info["rounds"])
            res[label] = {"value": sum(mc) / (sum(ms) * 1e-3) / 1e9, "unit": "GTEPS",
                                      "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                                      "steps_mean": statistics.mean(steps), "rounds_mean": statistics.mean(rounds)}
        out[name] = res
        del g, d, deg
        torch.cuda.empty_cache()
    return out


def serving(eic, torch, stream, rates, seconds_per_rate, max_per_rate):
    """Resident set of 8 graphs (RMAT scales 18..23, a second scale-22 seed, a
    2048^2 grid), Poisson request streams at each rate through eic_server_*;
    against one-at-a-time plain solves of the same requests (their measured
    service times replayed in arrival order)."""
    import numpy as np
    from paper_2506_19349_gb300 import graphgen

    t0 = time.perf_counter()
    wls = [graphgen.kron(s, seed=200 + s, nsources=1) for s in (18, 19, 20, 21, 22, 23)]
    wls.append(graphgen.kron(22, seed=300, nsources=1))
    wls.append(graphgen.road(2048, seed=301, wmax=255, nsources=1))
    gen_s = time.perf_counter() - t0
    graphs = [eic.Graph(w.n, w.src, w.dst, w.w) for w in wls]
    pools = [graphgen.pick_sources(w.n, w.src, w.dst, 32, 400 + k, "nonisolated") for k, w in enumerate(wls)]
    del wls
    # the request pool: 32 sources per graph; plain service time of each, on the device
    pool = [(g, int(s)) for g in range(len(graphs)) for s in pools[g]]
    dist = {g: eic.new_dist(graphs[g].n) for g in range(len(graphs))}
    svc = []
    for g, s in pool[:: len(pool) // 16]:  # warm-up
        eic.sssp(graphs[g], s, dist=dist[g])
    for g, s in pool:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        eic.sssp(graphs[g], s, dist=dist[g])
        e1.record(stream)
        e1.synchronize()
        svc.append(e0.elapsed_time(e1))
    plain_qps = 1000.0 / statistics.mean(svc)
    srv = eic.Server(graphs)
    t0 = time.perf_counter()
    shifts = srv.tune([pools[g][0] for g in range(len(graphs))])  # per-graph step width (exact)
    tune_s = time.perf_counter() - t0
    # like for like: the plain service time of each request at its graph's tuned step width
    svc_t = []
    for g, s in pool:
        p = eic.default_params(gap_shift=shifts[g])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        eic.sssp(graphs[g], s, dist=dist[g], params=p)
        e1.record(stream)
        e1.synchronize()
        svc_t.append(e0.elapsed_time(e1))
    plain_t_qps = 1000.0 / statistics.mean(svc_t)
    del dist
    rows = []
    rng = np.random.default_rng(11)
    switch = sys.getswitchinterval()
    sys.setswitchinterval(1e-4)  # the consumer thread releases results promptly
    for rate in rates:
        n_req = int(min(max_per_rate, max(50, rate * seconds_per_rate)))
        picks = rng.integers(len(pool), size=n_req)
        gaps = rng.exponential(1.0 / rate, size=n_req) if rate != float("inf") else np.zeros(n_req)
        arrive = np.cumsum(gaps)
        srv.reset_stats()
        tickets = []
        done_lat = []

        def consume():
            k = 0
            while k < n_req:
                if k >= len(tickets):
                    time.sleep(0.0002)
                    continue
                t = tickets[k]
                st = srv.wait(t, 600000)
                if st != 0:
                    raise RuntimeError(f"request status {st}")
                _, lat = srv.result(t, to_host=False)
                done_lat.append(lat)
                srv.release(t)
                k += 1

        th = threading.Thread(target=consume)
        th.start()
        start = time.perf_counter()
        for k in range(n_req):
            ahead = arrive[k] - (time.perf_counter() - start)
            if ahead > 3e-4:  # sleep (releasing the interpreter lock) until close to the arrival
                time.sleep(ahead - 2e-4)
            while time.perf_counter() - start < arrive[k]:
                pass
            g, s = pool[picks[k]]
            tickets.append(srv.submit(g, s))
        th.join()
        wall = time.perf_counter() - start
        st = srv.stats()
        def replay(times):  # one at a time: request k starts when it has arrived and k-1 is done
            fin, lat1 = 0.0, []
            for k in range(n_req):
                begin = max(arrive[k] * 1e3, fin)
                fin = begin + times[picks[k]]
                lat1.append(fin - arrive[k] * 1e3)
            lat1.sort()
            return {"qps": n_req / (fin * 1e-3), "p50_ms": lat1[len(lat1) // 2],
                    "p99_ms": lat1[min(len(lat1) - 1, int(0.99 * len(lat1)))]}

        dl = sorted(done_lat)
        svc_mix = [svc_t[picks[k]] for k in range(n_req)]
        rows.append({"rate_per_s": rate if rate != float("inf") else "all at once", "requests": n_req,
                     "served": {"qps": n_req / wall, "p50_ms": dl[len(dl) // 2],
                                "p99_ms": dl[min(len(dl) - 1, int(0.99 * len(dl)))],
                                "max_in_flight": st["max_in_flight"], "kernel_launches": st["kernel_launches"]},
                     "plain_service_tuned_ms": {"mean": statistics.mean(svc_mix),
                                                "p50": float(np.percentile(svc_mix, 50)),
                                                "p99": float(np.percentile(svc_mix, 99))},
                     "one_at_a_time": replay(svc), "one_at_a_time_tuned": replay(svc_t)})
    sys.setswitchinterval(switch)
    info = srv.stats()
    srv.close()
    best = max(r["served"]["qps"] for r in rows)
    return {"workload": "resident RMAT scales 18,19,20,21,22,22,23 and a 2048^2 grid (weights [1,255]); requests "
                        "(graph, source) uniform over 32 sources per graph, Poisson arrivals",
            "generate_s": gen_s, "groups": info["groups"], "blocks_per_group": info["blocks_per_group"],
            "tuned_gap_shift_per_graph": shifts, "tune_s": tune_s,
            "plain_one_at_a_time_qps": plain_qps, "plain_service_ms_mean": statistics.mean(svc),
            "plain_tuned_one_at_a_time_qps": plain_t_qps, "plain_tuned_service_ms_mean": statistics.mean(svc_t),
            "rates": rows, "peak_served_qps": best, "speedup_vs_one_at_a_time": best / plain_t_qps,
            "speedup_basis": "peak served queries/s vs one-at-a-time plain solves at the same per-graph step width",
            "speedup_vs_one_at_a_time_default_width": best / plain_qps,
            "latency": "submit to completion seen by the host runtime; one-at-a-time latencies replay the measured "
                       "plain service times of the same requests in arrival order"}


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2506_19349_gb300 import build as libbuild

    if not os.path.exists(os.path.join(ROOT, "paper_2506_19349_gb300", "libeic.so")):
        libbuild.build()
    import paper_2506_19349_gb300 as eic

    t0 = time.perf_counter()
    wl = make_workload(args.scale, args.sources, rank, args.road)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    n = g.n
    m_edges = g.m
    srcs = [int(s) for s in wl.sources]
    q = len(srcs)
    dists = [eic.new_dist(n) for _ in range(q)]
    # degrees for m_c (edges in the source's component)
    rowp = np.empty(n + 1, dtype=np.uint64)
    import ctypes

    eic.load_library().eic_graph_export(g.handle, rowp.ctypes.data, None, None, None)
    deg = torch.from_numpy(np.diff(rowp).astype(np.int64)).cuda()
    del rowp

    def run_step(collect=False):
        evs = []
        infos = []
        for i, s in enumerate(srcs):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, rc, info = eic.sssp(g, s, dist=dists[i], stats=collect)
            e1.record(stream)
            evs.append((e0, e1))
            infos.append(info)
        return evs, infos

    # warm-up (also yields m_c per source)
    for _ in range(max(args.warmup, 1)):
        run_step()
    torch.cuda.synchronize()
    m_c = [int(deg[d != -1].sum().item() // 2) for d in dists]
    edges_per_step = sum(m_c)

    # ---- timed region: device time with inputs resident
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    per_query = []
    all_infos = []
    for _ in range(args.steps):
        evs, infos = run_step(collect=True)
        per_query.append(evs)
        all_infos.extend(infos)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    total_ms = start.elapsed_time(end)
    q_ms = [a.elapsed_time(b) for evs in per_query for a, b in evs]
    total_ms = max_over_ranks(total_ms, world, "cuda")
    edges_all_ranks = sum_over_ranks(edges_per_step, world, "cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_gteps(edges_all_ranks, args.steps, total_ms)

    # roofline of the query kernel: algorithmic bytes per launch over its event duration
    b_alg = [16 * inf["frontier"] + 12 * inf["traversed"] + 8 * inf["improved"] + 12 * inf["pull_items"] + 4 * n
             for inf in all_infos]
    k_ms = [inf["kernel_ms"] for inf in all_infos]
    achieved = statistics.mean(b / (t * 1e-3) / 1e9 for b, t in zip(b_alg, k_ms))
    peak, peak_kind = peaks()

    # ---- end to end through the C ABI with host buffers: eic_sssp takes each
    # source id from the host and writes the distances into page-locked host
    # memory (its output kernel stores them across the host link); the result
    # is in host memory when the call returns
    e2e = None
    if not args.no_e2e:
        host_out = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
        for i, s in enumerate(srcs[:2]):  # warm-up; also checks the host copies against the device results
            eic.sssp(g, s, dist=host_out[i])
            if not torch.equal(host_out[i], dists[i].cpu()):
                raise RuntimeError("host-buffer result differs from the device-buffer result")
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        t_wall = time.perf_counter()
        e_start.record(stream)
        for _ in range(args.steps):
            for i, s in enumerate(srcs):
                eic.sssp(g, s, dist=host_out[i & 1])
        e_end.record(stream)
        torch.cuda.synchronize()
        wall_ms = (time.perf_counter() - t_wall) * 1e3
        e2e_ms = max_over_ranks(max(e_start.elapsed_time(e_end), wall_ms), world, "cuda")
        e2e = {"value": whole_job_gteps(edges_all_ranks, args.steps, e2e_ms), "unit": "GTEPS",
               "h2d_bytes_per_step": 4 * q, "d2h_bytes_per_step": 4 * n * q,
               "how": "eic_sssp per query with a page-locked host output array (host-to-device: the source id "
                      "passed to the call; device-to-host: n distances written by the output kernel)"}

    batched = None
    if not args.no_batched and world == 1:
        batched = {"same_workload": batched_same_workload(eic, torch, g, srcs, dists, stream, max(args.steps, 1),
                                                          value / world, edges_per_step)}
        del g, dists, deg
        torch.cuda.empty_cache()
        batched["mixed_32_graphs"] = batched_mixed(eic, torch, stream, max(args.steps, 1))
    served = None
    if not args.no_served and world == 1:
        torch.cuda.empty_cache()
        served = serving(eic, torch, stream, (100, 1000, 5000, 20000, float("inf")), 1.0, 2000)
    stressed = None
    if not args.no_stress and world == 1:
        torch.cuda.empty_cache()
        stressed = stress(eic, torch, stream, args.stress_sources)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, cpu_gteps, cpu_t = oracle_baseline(wl, args.cpu_sample, oracle_m_c)
        cpu = {"value": cpu_gteps, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_sample} binary-heap Dijkstra quer{'y' if args.cpu_sample == 1 else 'ies'} "
                         f"of the same kron{args.scale} workload on one host thread ({cpu_t:.1f} s; oracle CSR "
                         f"build untimed); host has {os.cpu_count()} cores"}

    if rank == 0:
        q_sorted = sorted(q_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(wl, args.scale, q, args.road) | {"m": int(m_edges), "m_c_mean": statistics.mean(m_c),
                                                            "build_s": build_s, "generate_s": gen_s},
            "latency_ms": {"p50": q_sorted[len(q_sorted) // 2], "p99": q_sorted[min(len(q_sorted) - 1,
                                                                                      int(0.99 * len(q_sorted)))],
                           "mean": statistics.mean(q_ms)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": None if args.road else MEASURED_TRAFFIC.get((args.scale, kernel_sources_sha256())),
                         "peak_kind": peak_kind,
                         "kernel": ("k_eic_fused" if args.road else "k_eic") +
                                   " (one launch per query; CUDA events around its launch)",
                         "kernel_ms_mean": statistics.mean(k_ms), "alg_bytes_mean": statistics.mean(b_alg)},
            "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e, "gpu_launches": 3 * q * args.steps,
            "counters_mean": {k: statistics.mean(inf[k] for inf in all_infos)
                              for k in ("steps", "rounds", "frontier", "traversed", "pulls", "improved", "heavy",
                                        "pull_items")},
            "batched": batched,
            "served": served,
            "stress": stressed,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
