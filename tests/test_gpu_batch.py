"""GPU parity of the batched path: every query of a persistent multi-query
launch equals the oracle's Dijkstra bit for bit, alone and in the mix, for
every group count, after CUDA-graph replay and after autotuning."""
import numpy as np
import pytest

import oracle as O
from paper_2506_19349_gb300 import graphgen as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_19349_gb300 as eic  # noqa: E402
from paper_2506_19349_gb300 import binding  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19349_gb300 import build

    build.build()


def _mixed_workloads():
    """Uneven sizes: Kronecker scales 9..14, grids 24..96, a uniform graph."""
    wls = [G.kron(9 + k, seed=60 + k, nsources=2) for k in range(6)]
    wls += [G.road(side, seed=70 + side, wmax=255, nsources=2) for side in (24, 48, 96)]
    wls.append(G.urand(12, 14, seed=80, nsources=2))
    return wls


@pytest.fixture(scope="module")
def mixed():
    graphs, srcs, want = [], [], []
    for wl in _mixed_workloads():
        g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
        og = O.Graph(wl.n, wl.src, wl.dst, wl.w)
        for s in wl.sources:
            graphs.append(g)
            srcs.append(int(s))
            want.append(og.dijkstra(int(s))[0])
    return graphs, srcs, want


def _check(dists, want):
    for i, (d, w) in enumerate(zip(dists, want)):
        got = eic.to_host_u32(d)
        assert np.array_equal(got, w), f"query {i}: {np.count_nonzero(got != w)} mismatches"


@pytest.mark.parametrize("groups", [1, 2, 3, 7, 64, 0])
def test_batch_every_group_count_is_exact(mixed, groups):
    graphs, srcs, want = mixed
    dists = [eic.new_dist(g.n) for g in graphs]
    for d in dists:
        d.fill_(7)  # every element must be written
    st = eic.sssp_batch(graphs, srcs, dists, params=eic.default_params(batch_groups=groups))
    assert (st == 0).all(), st
    _check(dists, want)


def test_batch_plan_replays_cuda_graph_and_tunes(mixed):
    graphs, srcs, want = mixed
    dists = [eic.new_dist(g.n) for g in graphs]
    b = eic.Batch(graphs, srcs, dists, params=eic.default_params(batch_groups=4))
    for rep in range(3):
        for d in dists:
            d.fill_(rep)
        b.run()
        st = b.wait()
        assert (st == 0).all(), st
        _check(dists, want)
    info = b.info()
    assert info["groups"] == 4 and info["queries"] == len(srcs)
    cfg = b.tune()
    assert cfg["groups"] >= 1 and cfg["tuned_ms"] > 0
    for d in dists:
        d.fill_(3)
    b.run()
    assert (b.wait() == 0).all()
    _check(dists, want)
    # each query's tuned step width, and the plain path at that width gives the same distances
    shifts = b.gap_shifts()
    assert len(shifts) == len(srcs) and max(shifts) <= 8 and max(shifts) == cfg["gap_shift"]
    for g, s, sh, w in zip(graphs, srcs, shifts, want):
        d, rc, _ = eic.sssp(g, s, params=eic.default_params(gap_shift=sh))
        assert rc == 0 and np.array_equal(eic.to_host_u32(d), w)
    b.close()


def test_batch_wide_weights_exact():
    """Weights of 2^20 and above (Function 2's exact sums, out of line in the
    batch kernel): every query equals Dijkstra for several group counts."""
    wl = G.kron(12, seed=92, weights=f"uniform:{1 << 24}", nsources=6)
    g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    og = O.Graph(wl.n, wl.src, wl.dst, wl.w)
    srcs = [int(s) for s in wl.sources]
    want = [og.dijkstra(s)[0] for s in srcs]
    for groups in (1, 3):
        dists = [eic.new_dist(g.n) for _ in srcs]
        st = eic.sssp_batch([g] * len(srcs), srcs, dists, params=eic.default_params(batch_groups=groups))
        assert (st == 0).all(), st
        _check(dists, want)


def test_batch_trivial_isolated_and_repeated_sources():
    # a graph without edges, an isolated source, the same source twice
    g0 = eic.Graph(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    src = np.array([0, 1, 1, 2], np.uint32)
    dst = np.array([1, 2, 3, 3], np.uint32)
    w = np.array([4, 1, 9, 2], np.uint32)
    g1 = eic.Graph(6, src, dst, w)
    og1 = O.Graph(6, src, dst, w)
    graphs = [g0, g1, g1, g1, g1]
    srcs = [3, 0, 5, 2, 2]
    dists = [eic.new_dist(g.n) for g in graphs]
    st = eic.sssp_batch(graphs, srcs, dists, params=eic.default_params(batch_groups=2))
    assert (st == 0).all()
    inf = eic.EIC_INF
    assert eic.to_host_u32(dists[0]).tolist() == [inf, inf, inf, 0, inf]
    assert eic.to_host_u32(dists[2]).tolist() == [inf] * 5 + [0]
    for k in (1, 3, 4):
        assert np.array_equal(eic.to_host_u32(dists[k]), og1.dijkstra(srcs[k])[0])


def test_batch_error_stops_only_its_group():
    # a 200-vertex path whose distances overflow, and small healthy graphs
    n = 200
    a = np.arange(n - 1, dtype=np.uint32)
    bad = eic.Graph(n, a, a + 1, np.full(n - 1, 100_000_000, np.uint32))
    wl = G.kron(8, seed=90, nsources=3)
    good = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    og = O.Graph(wl.n, wl.src, wl.dst, wl.w)
    srcs = [0] + [int(s) for s in wl.sources]
    graphs = [bad] + [good] * 3
    # two groups: the healthy queries finish on the other group
    dists = [eic.new_dist(g.n) for g in graphs]
    st = eic.sssp_batch(graphs, srcs, dists, params=eic.default_params(batch_groups=2))
    assert st[0] == binding.EOVERFLOW
    assert (st[1:] == 0).all(), st
    for k in range(1, 4):
        assert np.array_equal(eic.to_host_u32(dists[k]), og.dijkstra(srcs[k])[0])
    # one group, the failing query claimed first (largest graph): the rest is not run
    nb = 4 * good.m
    big = eic.Graph(nb, np.arange(nb - 1, dtype=np.uint32), np.arange(1, nb, dtype=np.uint32),
                    np.full(nb - 1, 100_000_000, np.uint32))
    assert big.m > good.m
    graphs = [big] + [good] * 3
    dists = [eic.new_dist(g.n) for g in graphs]
    st = eic.sssp_batch(graphs, srcs, dists, params=eic.default_params(batch_groups=1))
    assert st[0] == binding.EOVERFLOW
    assert (st[1:] == binding.EABORT).all(), st
    # the context and the scratch stay usable
    dists = [eic.new_dist(good.n) for _ in range(3)]
    st = eic.sssp_batch([good] * 3, srcs[1:], dists)
    assert (st == 0).all()
    for k in range(3):
        assert np.array_equal(eic.to_host_u32(dists[k]), og.dijkstra(srcs[k + 1])[0])


def test_batch_barrier_timeout_is_reported_and_context_survives():
    wl = G.kron(12, seed=91, nsources=4)
    g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    og = O.Graph(wl.n, wl.src, wl.dst, wl.w)
    srcs = [int(s) for s in wl.sources]
    dists = [eic.new_dist(g.n) for _ in srcs]
    st = eic.sssp_batch([g] * 4, srcs, dists, params=eic.default_params(batch_groups=2, max_spin_log2=1))
    assert set(st.tolist()) <= {binding.OK, binding.ETIMEOUT, binding.EABORT}
    st = eic.sssp_batch([g] * 4, srcs, dists, params=eic.default_params(batch_groups=2))
    assert (st == 0).all()
    for d, s in zip(dists, srcs):
        assert np.array_equal(eic.to_host_u32(d), og.dijkstra(s)[0])
