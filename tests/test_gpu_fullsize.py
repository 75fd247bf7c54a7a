"""Parity at the full sizes of the five workloads, on every source the bench
times, in the launch configurations it times them with.

The oracle's certificate (dist[s] = 0, no edge can improve a distance, every
reachable vertex has a tight incoming edge, reachability equals finiteness)
identifies the exact shortest distances at any size in O(m); it runs on host
threads, several sources at a time. Each workload also compares at least one
source in full with the oracle's Dijkstra, and one Kron 25 query's step trace
is recomputed from its exact distances (sumD, highD, Eq. 1-3, the settled
counts, termination and Function 2), which exercises the device's Eq. 2
(expm1, log1p) against the host's at full size.
"""
import gc

import numpy as np
import pytest

import oracle as O
from paper_2506_19349_gb300 import graphgen as G
from trace_check import check_trace_against_exact

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_19349_gb300 as eic  # noqa: E402

CHUNK = 16  # distance arrays held on the host at a time


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19349_gb300 import build

    build.build()


def _pair(wl):
    return eic.Graph(wl.n, wl.src, wl.dst, wl.w), O.Graph(wl.n, wl.src, wl.dst, wl.w)


def _certify(og, srcs, host_dists):
    res = og.check_many(srcs, host_dists)
    bad = [(s, r) for s, r in zip(srcs, res) if r != (0, 0)]
    assert not bad, bad


def _certify_plain(g, og, srcs, params=None):
    """Every source through eic_sssp (the bench's plain path), certified."""
    dists = [eic.new_dist(g.n) for _ in range(min(CHUNK, len(srcs)))]
    for c in range(0, len(srcs), CHUNK):
        part = srcs[c:c + CHUNK]
        for s, d in zip(part, dists):
            _, rc, _ = eic.sssp(g, s, dist=d, params=params)
            assert rc == 0, s
        _certify(og, part, [eic.to_host_u32(d).copy() for d in dists[:len(part)]])


@pytest.fixture(scope="module")
def kron25():
    """RMAT scale 25, edgefactor 16, weights [1,255]: the bench's 64 sources."""
    wl = G.kron(25, seed=2, nsources=64)
    g, og = _pair(wl)
    srcs = [int(s) for s in wl.sources]
    del wl
    gc.collect()
    yield g, og, srcs
    g.close()
    del og
    gc.collect()


def test_kron25_plain_every_source(kron25):
    g, og, srcs = kron25
    _certify_plain(g, og, srcs)
    # one source in full against Dijkstra, and its step trace against the exact distances
    d, rc, info = eic.sssp(g, srcs[0], trace_cap=4096)
    got = eic.to_host_u32(d)
    want, orc = og.dijkstra(srcs[0])
    assert rc == 0 and orc == 0 and np.array_equal(got, want)
    check_trace_against_exact(og, want, info["trace"])
    for r in info["trace"]:
        assert bool(r["flags"] & eic.STEP_PULL) == (r["st"] < r["lb"]), r


def test_kron25_batched_every_source(kron25):
    """All 64 sources as one tuned batch (the bench's same-workload batch)."""
    g, og, srcs = kron25
    dists = [eic.new_dist(g.n) for _ in srcs]
    b = eic.Batch([g] * len(srcs), srcs, dists)
    b.tune()
    for d in dists:
        d.fill_(7)
    b.run()
    assert (b.wait() == 0).all()
    b.close()
    for c in range(0, len(srcs), CHUNK):
        _certify(og, srcs[c:c + CHUNK], [eic.to_host_u32(d).copy() for d in dists[c:c + CHUNK]])
    del dists
    torch.cuda.empty_cache()


def test_road_4096_every_stress_source():
    """4096^2 grid, 10% of edges deleted, 2% diagonals, weights [1,4095]: the
    16 stress sources at the default step width and at gap_shift 4."""
    wl = G.road(4096, seed=3, wmax=4095, nsources=16)
    g, og = _pair(wl)
    srcs = [int(s) for s in wl.sources]
    for sh in (0, 4):
        _certify_plain(g, og, srcs, params=eic.default_params(gap_shift=sh))
    d, rc, _ = eic.sssp(g, srcs[0])
    want, orc = og.dijkstra(srcs[0])
    assert rc == 0 and orc == 0 and np.array_equal(eic.to_host_u32(d), want)


def test_kron25_lognormal_every_stress_source():
    """Scale-25 topology with log-normal weights (mu 3, sigma 1.5, clamped to [1,65535])."""
    wl = G.kron(25, seed=2, weights="lognormal", nsources=16)
    g, og = _pair(wl)
    srcs = [int(s) for s in wl.sources]
    del wl
    gc.collect()
    _certify_plain(g, og, srcs)
    d, rc, _ = eic.sssp(g, srcs[0])
    want, orc = og.dijkstra(srcs[0])
    assert rc == 0 and orc == 0 and np.array_equal(eic.to_host_u32(d), want)


def test_batch_set_tuned_plan():
    """32 graphs of uneven size x 8 sources through a tuned, graph-replayed batch plan."""
    wls = G.batch_set()
    graphs, oracles, srcs, gi = [], [], [], []
    for k, wl in enumerate(wls):
        g, og = _pair(wl)
        graphs.append(g)
        oracles.append(og)
        for s in wl.sources:
            srcs.append(int(s))
            gi.append(k)
    del wls
    dists = [eic.new_dist(graphs[k].n) for k in gi]
    b = eic.Batch([graphs[k] for k in gi], srcs, dists)
    b.tune()
    for d in dists:
        d.fill_(7)
    b.run()
    assert (b.wait() == 0).all()
    for k, s, d in zip(gi, srcs, dists):
        assert oracles[k].check(s, eic.to_host_u32(d)) == (0, 0), (k, s)
    b.close()


def test_serving_set_every_pool_source():
    """Resident RMAT scales 18..23 (and a second scale-22 seed) and a 2048^2
    grid, with the per-graph step widths the server's tuner picks: every
    source of the bench's request pool (32 per graph), in flight together."""
    wls = [G.kron(s, seed=200 + s, nsources=1) for s in (18, 19, 20, 21, 22, 23)]
    wls.append(G.kron(22, seed=300, nsources=1))
    wls.append(G.road(2048, seed=301, wmax=255, nsources=1))
    pairs = [_pair(w) for w in wls]
    pools = [G.pick_sources(w.n, w.src, w.dst, 32, 400 + k, "nonisolated") for k, w in enumerate(wls)]
    reqs = [(k, int(s)) for k in range(len(wls)) for s in pools[k]]
    del wls
    srv = eic.Server([p[0] for p in pairs])
    srv.tune([int(pools[k][0]) for k in range(len(pairs))])
    tickets = [srv.submit(k, s) for k, s in reqs]
    got = {}
    for t, (k, s) in zip(tickets, reqs):
        assert srv.wait(t) == 0
        got[(k, s)] = srv.result(t, pairs[k][0].n)[0]
        srv.release(t)
    srv.close()
    for k in range(len(pairs)):
        srcs = [s for kk, s in reqs if kk == k]
        _certify(pairs[k][1], srcs, [got[(k, s)] for s in srcs])
