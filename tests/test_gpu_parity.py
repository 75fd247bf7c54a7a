"""GPU parity: libeic against the CPU oracle, element by element.

Distances are uint32 and must match Dijkstra bit for bit. The device CSR must
equal the oracle's CSR byte for byte; RtoW and highD(0) must match exactly;
the per-step trace <lb, ub, st> with its statistics must equal the oracle's
sequential Algorithm 1 (every quantity is a function of the exact distances).
"""
import ctypes

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


def _pair(wl):
    return eic.Graph(wl.n, wl.src, wl.dst, wl.w), O.Graph(wl.n, wl.src, wl.dst, wl.w)


def _cases():
    yield "urand14", G.urand(14, 17, seed=1, nsources=4)
    yield "urand12_sparse", G.urand(12, 12, seed=8, nsources=4)
    yield "kron10", G.kron(10, seed=20, nsources=4)
    yield "kron14", G.kron(14, seed=21, nsources=4)
    yield "kron16", G.kron(16, seed=2, nsources=3)
    yield "kron13_lognormal", G.kron(13, seed=22, weights="lognormal", nsources=3)
    yield "grid64", G.road(64, seed=23, wmax=4095, nsources=3)
    yield "grid128_w255", G.road(128, seed=24, wmax=255, nsources=2)
    w = G.kron(12, seed=25, nsources=3)
    w.w = np.ones_like(w.w)
    yield "kron12_unit", w
    w = G.kron(12, seed=26, nsources=3)
    w.w = (w.w % 3 + 1).astype(np.uint32)
    yield "kron12_w123", w
    # the paper's weight variants (Eq. 7 power, Eq. 8 pivot)
    for p in (1, 4, 10):
        yield f"kron12_power{p}", G.kron(12, seed=27, weights=f"power:{p}", nsources=2)
    for y in (0.1, 0.9):
        yield f"kron12_pivot{y}", G.kron(12, seed=28, weights=f"pivot:{y}", nsources=2)
    # weights of 2^20 and above: Function 2 sums D(x') exactly from the settled list
    for wmax, scale, seed in ((1 << 21, 12, 90), (1 << 24, 12, 90), (1 << 27, 13, 91)):
        yield f"kron{scale}_uniform{wmax}", G.kron(scale, seed=seed, weights=f"uniform:{wmax}", nsources=3)
    yield "kron13_power24", G.kron(13, seed=91, weights="power:24", nsources=3)


CASES = list(_cases())


@pytest.mark.parametrize("name,wl", CASES, ids=[c[0] for c in CASES])
def test_csr_equals_oracle(name, wl):
    g, og = _pair(wl)
    row, nbr, w, rt = g.export()
    orow, onbr, ow = og.csr()
    assert np.array_equal(row, orow)
    assert np.array_equal(nbr, onbr)
    assert np.array_equal(w, ow)
    assert np.array_equal(rt, og.rtow())
    assert g.highd0 == O.highd(og.degrees())
    assert (g.m, g.max_w, g.max_deg) == (og.m, og.maxw, og.maxdeg)


@pytest.mark.parametrize("name,wl", CASES, ids=[c[0] for c in CASES])
def test_device_row_order(name, wl):
    """The CSR as the kernels read it: internal ids are the non-isolated
    vertices by (degree descending, original id), each row is strictly
    increasing in (weight, the neighbour's original id) (the window searches
    rely on the weight order of Section 4.1), and every row holds the
    oracle's edges."""
    g, og = _pair(wl)
    i2o, row, nbr, w = g.export_internal()
    orow, onbr, ow = og.csr()
    deg = np.diff(orow).astype(np.int64)
    want_ids = np.lexsort((np.arange(wl.n), -deg))[: int((deg > 0).sum())]
    assert np.array_equal(i2o, want_ids.astype(np.uint32))
    assert row[0] == 0 and row[-1] == nbr.size and np.all(np.diff(row.astype(np.int64)) >= 1)
    assert np.array_equal(np.diff(row.astype(np.int64)), deg[i2o])
    key = (w.astype(np.uint64) << np.uint64(32)) | i2o[nbr].astype(np.uint64)
    inrow = np.ones(max(nbr.size - 1, 0), dtype=bool)  # entry pairs (k, k + 1) of the same row
    inrow[row[1:-1].astype(np.int64) - 1] = False
    assert np.all(key[1:][inrow] > key[:-1][inrow]), "a row is not sorted by (weight, original neighbour id)"
    for i in range(0, i2o.size, max(1, i2o.size // 257)):  # rows back in the caller's ids, against the oracle
        u = i2o[i]
        got = sorted(zip(w[row[i]:row[i + 1]].tolist(), i2o[nbr[row[i]:row[i + 1]]].tolist()))
        want = sorted(zip(ow[orow[u]:orow[u + 1]].tolist(), onbr[orow[u]:orow[u + 1]].tolist()))
        assert got == want, (name, int(u))


@pytest.mark.parametrize("name,wl", CASES, ids=[c[0] for c in CASES])
def test_distances_bit_exact_and_trace(name, wl):
    g, og = _pair(wl)
    for s in wl.sources:
        s = int(s)
        dist, rc, info = eic.sssp(g, s, trace_cap=4096)
        got = eic.to_host_u32(dist)
        want, orc = og.dijkstra(s)
        assert rc == 0 and orc == 0
        mism = np.flatnonzero(got != want)
        assert mism.size == 0, f"{name} s={s}: {mism.size} mismatches, first {mism[:5]} got {got[mism[:5]]} " \
                               f"want {want[mism[:5]]}"
        assert og.check(s, got) == (0, 0)
        _, _, otrace, otot = og.eic(s)
        keys = ("lb", "ub", "st", "gap_lb", "sumd_lb", "highd_lb", "settled")
        gt = [{k: r[k] for k in keys} for r in info["trace"]]
        ot = [{k: r[k] for k in keys} for r in otrace]
        assert gt == ot, f"{name} s={s}: trace differs at step {next(i for i, (a, b) in enumerate(zip(gt, ot)) if a != b) if len(gt) == len(ot) else 'len'}"
        assert info["steps"] == otot["steps"]
        # the pull ran exactly in the steps with st < lb (Function 1), and only a pull is swept
        for r in info["trace"]:
            assert bool(r["flags"] & eic.STEP_PULL) == (r["st"] < r["lb"]), (name, s, r)
            assert not (r["flags"] & eic.STEP_SWEPT) or r["flags"] & eic.STEP_PULL, (name, s, r)


def test_sweep_and_listed_pulls_both_exercised():
    """On Kronecker graphs both pull forms run and stay exact: the compacted
    vertex-order sweep (every pull step of the smaller graphs) and the listed
    pull over a prefix of the weight-ordered vertices (a step of one Kron 18
    source, whose pull set holds fewer than half of the vertices)."""
    kinds = set()
    for scale, seed, weights in ((14, 21, "uniform255"), (13, 22, "lognormal"), (18, 2, "uniform255")):
        wl = G.kron(scale, seed=seed, weights=weights, nsources=3)
        g, og = _pair(wl)
        for s in wl.sources:
            dist, rc, info = eic.sssp(g, int(s), trace_cap=4096)
            assert rc == 0
            assert np.array_equal(eic.to_host_u32(dist), og.dijkstra(int(s))[0])
            for r in info["trace"]:
                if r["flags"] & eic.STEP_PULL:
                    kinds.add("swept" if r["flags"] & eic.STEP_SWEPT else "listed")
    assert kinds == {"swept", "listed"}, kinds


def test_parent_output():
    wl = G.kron(12, seed=30, nsources=2)
    g, og = _pair(wl)
    for s in wl.sources:
        par = torch.empty(wl.n, dtype=torch.int32, device="cuda")
        dist, rc, _ = eic.sssp(g, int(s), parent=par)
        d = eic.to_host_u32(dist)
        assert np.array_equal(eic.to_host_u32(par), og.parent(int(s), d))


def test_fused_rounds_exact_with_fewer_rounds():
    """Graphs whose degrees are all <= heavy_min run fused rounds (bucket
    fusion): the distances and the step trace equal the oracle's, with or
    without fusion, and fusion takes fewer grid-wide rounds."""
    for wl in (G.road(96, seed=35, wmax=4095, nsources=2), G.road(128, seed=36, wmax=255, nsources=2)):
        g, og = _pair(wl)
        assert g.max_deg <= 32
        for s in wl.sources:
            s = int(s)
            want, _ = og.dijkstra(s)
            _, _, otrace, _ = og.eic(s)
            keys = ("lb", "ub", "st", "gap_lb", "sumd_lb", "highd_lb", "settled")
            rounds = []
            for p in (None, eic.default_params(flags=eic.FLAG_NO_FUSE)):
                d, rc, info = eic.sssp(g, s, params=p, stats=True, trace_cap=1 << 14)
                assert rc == 0 and np.array_equal(eic.to_host_u32(d), want)
                assert [{k: r[k] for k in keys} for r in info["trace"]] == [{k: r[k] for k in keys} for r in otrace]
                rounds.append(info["rounds"])
            assert rounds[0] < rounds[1], rounds


def test_fused_rounds_local_queue_overflow():
    """Degree-24 graphs (a union of random perfect matchings, unit and small
    weights): a warp's wave improves more vertices than its local queue holds,
    and the rest goes to the next round's queue; still exact."""
    rng = np.random.default_rng(37)
    n, k = 8192, 24
    src, dst = [], []
    for _ in range(k):
        perm = rng.permutation(n).astype(np.uint32)
        src.append(perm[0::2])
        dst.append(perm[1::2])
    src, dst = np.concatenate(src), np.concatenate(dst)
    for w in (np.ones(src.size, np.uint32), rng.integers(1, 9, src.size).astype(np.uint32)):
        g = eic.Graph(n, src, dst, w)
        og = O.Graph(n, src, dst, w)
        assert g.max_deg <= 32
        for s in (0, 4097):
            d, rc, _ = eic.sssp(g, s)
            assert rc == 0 and np.array_equal(eic.to_host_u32(d), og.dijkstra(s)[0])


def test_output_alignment_and_ragged_tail():
    """The output kernel writes 16-byte groups when dist is 16-byte aligned and
    one value at a time otherwise; n = 4k + 3 leaves a ragged tail."""
    n = 4 * 257 + 3
    src = np.arange(n - 1, dtype=np.uint32)
    w = (src % 5 + 1).astype(np.uint32)
    extra_s = np.array([0, 10, 500], np.uint32)
    extra_d = np.array([n - 1, n - 2, n - 5], np.uint32)
    s_all, d_all = np.concatenate([src, extra_s]), np.concatenate([src + 1, extra_d])
    w_all = np.concatenate([w, np.array([7, 3, 11], np.uint32)])
    g = eic.Graph(n, s_all, d_all, w_all)
    og = O.Graph(n, s_all, d_all, w_all)
    for s in (0, n - 1, n - 3):
        want, _ = og.dijkstra(s)
        for off in (0, 1, 3):
            buf = torch.full((n + 4,), 7, dtype=torch.int32, device="cuda")
            d = buf[off:off + n]
            _, rc, _ = eic.sssp(g, s, dist=d)
            assert rc == 0 and np.array_equal(eic.to_host_u32(d), want), (s, off)
            assert (buf[:off] == 7).all() and (buf[off + n:] == 7).all()


def test_host_output_arrays():
    """dist and parent in page-locked host memory are written directly by the
    query; pageable host memory is rejected before any launch."""
    wl = G.kron(12, seed=34, nsources=2)
    g, og = _pair(wl)
    for s in wl.sources:
        s = int(s)
        d = torch.empty(wl.n, dtype=torch.int32).pin_memory()
        p = torch.empty(wl.n, dtype=torch.int32).pin_memory()
        d.fill_(7)
        _, rc, _ = eic.sssp(g, s, dist=d, parent=p)
        want, _ = og.dijkstra(s)
        assert rc == 0 and np.array_equal(d.numpy().view(np.uint32), want)
        assert np.array_equal(p.numpy().view(np.uint32), og.parent(s, want))
    pageable = torch.empty(wl.n, dtype=torch.int32)
    _, rc, _ = eic.sssp(g, int(wl.sources[0]), dist=pageable, raise_on_error=False)
    assert rc == binding.EINVAL
    dev = eic.new_dist(wl.n)
    _, rc, _ = eic.sssp(g, int(wl.sources[0]), dist=dev, parent=pageable, raise_on_error=False)
    assert rc == binding.EINVAL
    # a graph without edges, host output
    g0 = eic.Graph(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    d = torch.empty(5, dtype=torch.int32).pin_memory()
    _, rc, _ = eic.sssp(g0, 3, dist=d)
    assert rc == 0 and d.numpy().view(np.uint32).tolist() == [eic.EIC_INF] * 3 + [0, eic.EIC_INF]


def test_no_pull_and_step_scaling_stay_exact():
    wl = G.kron(14, seed=31, nsources=2)
    g, og = _pair(wl)
    for s in wl.sources:
        want, _ = og.dijkstra(int(s))
        for p in (eic.default_params(flags=eic.FLAG_NO_PULL), eic.default_params(gap_shift=2),
                  eic.default_params(heavy_min=16), eic.default_params(heavy_min=4096), eic.default_params(block_threads=256), eic.default_params(block_threads=128),
                  eic.default_params(st_num=7)):
            dist, rc, _ = eic.sssp(g, int(s), params=p)
            assert np.array_equal(eic.to_host_u32(dist), want)


def test_edge_cases():
    # single vertex, no edges
    g = eic.Graph(1, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    d, rc, _ = eic.sssp(g, 0)
    assert eic.to_host_u32(d).tolist() == [0]
    # self-loops and duplicates only around an isolated source
    src = np.array([0, 1, 1, 2, 2], np.uint32)
    dst = np.array([0, 2, 2, 1, 3], np.uint32)
    w = np.array([5, 9, 4, 7, 1], np.uint32)
    g = eic.Graph(5, src, dst, w)
    d, _, _ = eic.sssp(g, 0)
    assert eic.to_host_u32(d).tolist() == [0, eic.EIC_INF, eic.EIC_INF, eic.EIC_INF, eic.EIC_INF]
    d, _, _ = eic.sssp(g, 1)
    assert eic.to_host_u32(d).tolist() == [eic.EIC_INF, 0, 4, 5, eic.EIC_INF]
    # long path: many rounds in one step
    n = 3000
    src = np.arange(n - 1, dtype=np.uint32)
    g = eic.Graph(n, src, src + 1, (src % 7 + 1).astype(np.uint32))
    d, _, _ = eic.sssp(g, 0)
    assert np.array_equal(eic.to_host_u32(d), np.concatenate([[0], np.cumsum(src % 7 + 1)]).astype(np.uint32))
    # star: hub source (the first step's ub becomes 0) and leaf source
    n = 5000
    leaves = np.arange(1, n, dtype=np.uint32)
    ww = (leaves % 250 + 1).astype(np.uint32)
    g = eic.Graph(n, np.zeros(n - 1, np.uint32), leaves, ww)
    og = O.Graph(n, np.zeros(n - 1, np.uint32), leaves, ww)
    for s in (0, 17, n - 1):
        d, _, _ = eic.sssp(g, s)
        assert np.array_equal(eic.to_host_u32(d), og.dijkstra(s)[0])


def test_hub_sources_kron():
    wl = G.kron(15, seed=32, nsources=1)
    g, og = _pair(wl)
    deg = og.degrees()
    for s in np.argsort(deg)[-3:]:  # highest-degree vertices: deg(s) >= highD(0)
        d, _, info = eic.sssp(g, int(s), trace_cap=256)
        assert np.array_equal(eic.to_host_u32(d), og.dijkstra(int(s))[0])
        assert info["trace"][0]["ub"] == 0


def test_errors():
    wl = G.urand(10, 12, seed=3)
    g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    _, rc, _ = eic.sssp(g, wl.n, raise_on_error=False)
    assert rc == binding.EINVAL
    with pytest.raises(eic.EicError) as e:
        eic.Graph(4, np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), np.array([3, 0], np.uint32))
    assert e.value.status == binding.EINVAL
    with pytest.raises(eic.EicError):
        eic.Graph(4, np.array([0, 1], np.uint32), np.array([1, 4], np.uint32), np.array([3, 1], np.uint32))
    # overflow: the largest distance plus the largest weight reaches 2^32-1
    w = np.array([2_000_000_000, 2_000_000_000, 200_000_000], np.uint32)
    g = eic.Graph(4, np.arange(3, dtype=np.uint32), np.arange(1, 4, dtype=np.uint32), w)
    _, rc, _ = eic.sssp(g, 0, raise_on_error=False)
    assert rc == binding.EOVERFLOW
    w2 = np.array([1_000_000_000, 1_000_000_000, 100], np.uint32)
    g = eic.Graph(4, np.arange(3, dtype=np.uint32), np.arange(1, 4, dtype=np.uint32), w2)
    d, rc, _ = eic.sssp(g, 0)
    assert eic.to_host_u32(d).tolist() == [0, 1_000_000_000, 2_000_000_000, 2_000_000_100]


def test_barrier_timeout_is_reported_and_context_survives():
    wl = G.kron(12, seed=33, nsources=1)
    g, og = _pair(wl)
    p = eic.default_params(max_spin_log2=1)  # two polls: waiting blocks give up at once
    _, rc, _ = eic.sssp(g, int(wl.sources[0]), params=p, raise_on_error=False)
    assert rc in (binding.ETIMEOUT, binding.OK)
    d, rc, _ = eic.sssp(g, int(wl.sources[0]))
    assert rc == 0 and np.array_equal(eic.to_host_u32(d), og.dijkstra(int(wl.sources[0]))[0])


def test_batch_equals_single_queries():
    wls = [G.kron(11, seed=40, nsources=3), G.road(48, seed=41, wmax=255, nsources=3), G.urand(11, 14, seed=42,
                                                                                                 nsources=3)]
    graphs, srcs, dists, want = [], [], [], []
    for wl in wls:
        g, og = _pair(wl)
        for s in wl.sources:
            graphs.append(g)
            srcs.append(int(s))
            dists.append(eic.new_dist(wl.n))
            want.append(og.dijkstra(int(s))[0])
    st = eic.sssp_batch(graphs, srcs, dists)
    assert (st == 0).all()
    for d, w in zip(dists, want):
        assert np.array_equal(eic.to_host_u32(d), w)


def test_counters_in_paper_bands():
    wl = G.kron(16, seed=2, nsources=2)
    g, og = _pair(wl)
    for s in wl.sources:
        d, _, info = eic.sssp(g, int(s), stats=True)
        reach = int((eic.to_host_u32(d) != eic.EIC_INF).sum())
        assert info["frontier"] / reach <= 1.2
        assert 2.0 <= info["traversed"] / reach <= 7.0
