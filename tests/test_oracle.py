"""Pins for the CPU oracle (no GPU).

The oracle is pinned to things other than itself: brute force (Bellman-Ford,
Floyd-Warshall on the raw tuples, exhaustive tiny topologies), closed forms
(BFS hop counts, prefix sums, Manhattan distance, stars, components), an
invariant certificate that must reject mutated arrays, values printed by the
paper (Table 1 highD(0)), exact rational definitions of the RtoW quantile and
of highD, the inverse identity of Eq. 2, and the paper's exactness claim for
Algorithm 1 (its distances equal Dijkstra's on every input).
"""
import itertools
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2506_19349_gb300 import graphgen as G
from trace_check import check_trace_against_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _rand_tuples(rng, n, ne, wvals, loops=True, dups=True):
    src, dst, w = [], [], []
    for _ in range(ne):
        a, b = rng.randrange(n), rng.randrange(n)
        if a == b and not loops:
            continue
        src.append(a)
        dst.append(b)
        w.append(rng.choice(wvals))
        if dups and rng.random() < 0.2:
            src.append(b)
            dst.append(a)
            w.append(rng.choice(wvals))
    return (np.array(src, dtype=np.uint32), np.array(dst, dtype=np.uint32), np.array(w, dtype=np.uint32))


# ---------------------------------------------------------------- CSR builder

def test_csr_builder_matches_dict_construction():
    rng = random.Random(5)
    for trial in range(40):
        n = rng.randrange(1, 40)
        src, dst, w = _rand_tuples(rng, n, rng.randrange(0, 120), [1, 2, 3, 7, 100])
        g = O.Graph(n, src, dst, w)
        row, nbr, ww = g.csr()
        best = {}
        for a, b, x in zip(src.tolist(), dst.tolist(), w.tolist()):
            if a == b:
                continue
            k = (min(a, b), max(a, b))
            best[k] = min(best.get(k, 1 << 40), x)
        rows = {u: [] for u in range(n)}
        for (a, b), x in best.items():
            rows[a].append((x, b))
            rows[b].append((x, a))
        assert g.nnz == 2 * len(best)
        for u in range(n):
            got = list(zip(ww[row[u]:row[u + 1]].tolist(), nbr[row[u]:row[u + 1]].tolist()))
            assert got == sorted(rows[u]), (trial, u)


def test_csr_builder_rejects_bad_tuples():
    with pytest.raises(O.OracleError):
        O.Graph(3, [0], [3], [1])
    with pytest.raises(O.OracleError):
        O.Graph(3, [0], [1], [0])


# ------------------------------------------------- brute force on tiny graphs

def test_exhaustive_tiny_topologies_dijkstra_bf_fw():
    rng = random.Random(11)
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        src = np.array([a for a, _ in es], dtype=np.uint32)
        dst = np.array([b for _, b in es], dtype=np.uint32)
        w = np.array([rng.choice([1, 2, 3]) for _ in es], dtype=np.uint32)
        g = O.Graph(n, src, dst, w)
        for s in range(n):
            d, rc = g.dijkstra(s)
            assert rc == 0
            bf, rc2 = O.bellman_ford(n, src, dst, w, s)
            fw = O.floyd_warshall(n, src, dst, w, s)
            assert (d == bf).all() and (d == fw).all(), (mask, s)
            assert g.check(s, d) == (0, 0)


def test_random_small_graphs_with_ties_dijkstra_bf_fw():
    rng = random.Random(12)
    for trial in range(60):
        n = rng.randrange(2, 65)
        src, dst, w = _rand_tuples(rng, n, rng.randrange(0, 3 * n), [1, 2, 3])
        g = O.Graph(n, src, dst, w)
        s = rng.randrange(n)
        d, rc = g.dijkstra(s)
        bf, _ = O.bellman_ford(n, src, dst, w, s)
        fw = O.floyd_warshall(n, src, dst, w, s)
        assert (d == bf).all() and (d == fw).all(), trial
        assert g.check(s, d) == (0, 0)


# ---------------------------------------------------------------- closed forms

def test_unit_weights_equal_bfs_hops():
    w = G.urand(12, 15, seed=3)
    ones = np.ones_like(w.w)
    g = O.Graph(w.n, w.src, w.dst, ones)
    row, nbr, _ = g.csr()
    s = int(w.sources[0])
    hops = np.full(w.n, O.INF, dtype=np.uint64)
    hops[s] = 0
    q = [s]
    for u in q:
        for v in nbr[row[u]:row[u + 1]]:
            if hops[v] == O.INF:
                hops[v] = hops[u] + 1
                q.append(int(v))
    d, _ = g.dijkstra(s)
    assert (d.astype(np.uint64) == hops).all()


def test_path_graph_prefix_sums():
    rng = np.random.default_rng(4)
    n = 500
    w = rng.integers(1, 1000, size=n - 1).astype(np.uint32)
    src = np.arange(n - 1, dtype=np.uint32)
    dst = src + 1
    g = O.Graph(n, src, dst, w)
    d, _ = g.dijkstra(0)
    assert (d == np.concatenate([[0], np.cumsum(w)])).all()
    d, _ = g.dijkstra(n - 1)
    assert (d == np.concatenate([np.cumsum(w[::-1])[::-1], [0]])).all()


def test_unit_grid_manhattan():
    k = 37
    src, dst = G.grid(k, 0.0, 0.0, 1)
    g = O.Graph(k * k, src, dst, np.ones_like(src))
    s = 5 * k + 11
    d, _ = g.dijkstra(s)
    r, c = np.divmod(np.arange(k * k), k)
    assert (d == np.abs(r - 5) + np.abs(c - 11)).all()


def test_star_and_components():
    n = 50
    src = np.zeros(n - 1 - 10, dtype=np.uint32)
    dst = np.arange(1, n - 10, dtype=np.uint32)
    w = (dst * 7 % 13 + 1).astype(np.uint32)
    # second component on vertices n-10..n-1: a path
    src2 = np.arange(n - 10, n - 1, dtype=np.uint32)
    g = O.Graph(n, np.concatenate([src, src2]), np.concatenate([dst, src2 + 1]),
                np.concatenate([w, np.full(9, 5, np.uint32)]))
    d, _ = g.dijkstra(0)
    assert d[0] == 0 and (d[1:n - 10] == w).all() and (d[n - 10:] == O.INF).all()
    leaf = 3
    d2, _ = g.dijkstra(leaf)
    assert d2[0] == w[leaf - 1]
    assert all(d2[v] == w[leaf - 1] + w[v - 1] for v in range(1, n - 10) if v != leaf)


# ------------------------------------------------------------ invariant check

def test_checker_rejects_mutations():
    w = G.urand(11, 14, seed=9)
    g = O.Graph(w.n, w.src, w.dst, w.w)
    s = int(w.sources[0])
    d, _ = g.dijkstra(s)
    assert g.check(s, d) == (0, 0)
    rng = np.random.default_rng(0)
    finite = np.flatnonzero((d != O.INF) & (np.arange(w.n) != s))
    for v in rng.choice(finite, 30, replace=False):
        for delta in (-1, 1, 7):
            e = d.copy()
            e[v] = int(d[v]) + delta
            code, _ = g.check(s, e)
            assert code in (2, 3), (v, delta)
        e = d.copy()
        e[v] = O.INF
        assert g.check(s, e)[0] in (2, 4)
    e = d.copy()
    e[s] = 1
    assert g.check(s, e)[0] == 1


def test_overflow_contract():
    # path whose last distance plus maxW reaches 2^32 - 1
    w = np.array([2_000_000_000, 2_000_000_000, 200_000_000], dtype=np.uint32)
    g = O.Graph(4, np.arange(3, dtype=np.uint32), np.arange(1, 4, dtype=np.uint32), w)
    _, rc = g.dijkstra(0)
    assert rc == 3
    _, rc, _, _ = g.eic(0)
    assert rc == 3
    w2 = np.array([1_000_000_000, 1_000_000_000, 100], dtype=np.uint32)
    g2 = O.Graph(4, np.arange(3, dtype=np.uint32), np.arange(1, 4, dtype=np.uint32), w2)
    d, rc = g2.dijkstra(0)
    assert rc == 0 and d[3] == 2_000_000_100
    de, rc, _, _ = g2.eic(0)
    assert rc == 0 and (de == d).all()


# ------------------------------------------------------------------ statistics

def _rtow_by_definition(weights, R):
    ws = sorted(weights)
    m = len(ws)
    out = []
    for i in range(R):
        ratio = Fraction(i, R - 1)
        # smallest W in the multiset with P(w <= W) >= ratio
        out.append(next(W for W in ws if Fraction(sum(1 for x in ws if x <= W), m) >= ratio))
    return out


def test_rtow_matches_quantile_definition():
    rng = random.Random(3)
    for trial in range(30):
        m = rng.randrange(1, 60)
        ws = [rng.choice([1, 2, 5, 9, 200, 255]) if trial % 2 else rng.randrange(1, 10_000) for _ in range(m)]
        for R in (2, 3, 7, 16):
            assert O.rtow(ws, R).tolist() == _rtow_by_definition(ws, R), (trial, R)
    t = O.rtow(list(range(1, 256)), 4096)
    assert t[0] == 1 and t[-1] == 255


def _highd_brute(degs):
    """min over thresholds t in present degrees of |sum(deg<t) - sum(deg>=t)|, smallest t on ties."""
    degs = [d for d in degs if d > 0]
    if not degs:
        return 0
    best = None
    for t in sorted(set(degs)):
        low = sum(d for d in degs if d < t)
        high = sum(d for d in degs if d >= t)
        if best is None or abs(high - low) < best[0]:
            best = (abs(high - low), t)
    return best[1]


def test_highd_matches_brute_force():
    rng = random.Random(8)
    for trial in range(200):
        k = rng.randrange(0, 40)
        degs = [rng.choice([0, 1, 1, 2, 3, 5, 8, 40, 300]) for _ in range(k)]
        assert O.highd(degs) == _highd_brute(degs), degs
    assert O.highd([6] * 20) == 6  # regular: the only candidate
    assert O.highd([1] * 10 + [10]) == 10  # L=10 vs H=10


def test_highd_table1_urand():
    """Table 1: Urand (average degree 32) has highD(0) = 33."""
    gold = _golden("table1_urand_highd.txt")
    for ln in (15, 17):
        src, dst = G.uniform(1 << ln, 1 << (ln + 4), 11 + ln)
        g = O.Graph(1 << ln, src, dst, np.ones_like(src))
        deg = g.degrees()
        assert abs(deg.mean() - gold["avg_degree"]) < 1e-9
        assert O.highd(deg) == gold["highd0"]


def test_highd_table1_road_like():
    """Table 1: Road (average degree 2.44) has highD(0) = 3; a grid keeping 61%
    of its edges has the same average degree."""
    gold = _golden("table1_road_highd.txt")
    src, dst = G.grid(400, 0.39, 0.0, 21)
    g = O.Graph(400 * 400, src, dst, np.ones_like(src))
    deg = g.degrees()
    assert abs(deg.mean() - gold["avg_degree"]) < 0.02
    assert O.highd(deg) == gold["highd0"]


def test_gap_eq2_inverse_identity_and_branches():
    R = 4096
    rt = np.arange(1, R + 1, dtype=np.uint32)  # RtoW[i] = i + 1 exposes the index
    two_m = 1_000_000
    for highd in (4, 5, 17, 33, 300, 2517):
        for sumd in (two_m, 900_000, 500_000, 300_000, 10, 0):
            g, idx, ratio = O.gap(sumd, highd, two_m, rt)
            frac = max(sumd, two_m - sumd) / two_m
            prob = min(0.9, frac)
            assert prob >= 0.5
            # (1 - ratio)^(prob * highD) = 1 - prob  (Eq. 2 solved for 1 - prob)
            assert math.isclose((1 - ratio) ** (prob * highd), 1 - prob, rel_tol=1e-12)
            assert idx == math.floor(ratio * (R - 1)) and g == idx + 1
    for highd in (0, 1, 2, 3):  # Eq. 3 first branch, alpha = 3 inclusive
        g, idx, _ = O.gap(123, highd, two_m, rt)
        assert g == R and idx == R - 1
    gs = [O.gap(two_m, h, two_m, rt)[0] for h in (4, 8, 16, 64, 256, 1024)]
    assert gs == sorted(gs, reverse=True)  # larger highD -> smaller step


def test_profit_special_cases():
    maxw, two_m = 255, 10_000
    lb, y = 1000, 1010
    # no settled degree in [x', lb): nothing pushed, profit = -pulled <= 0
    assert O.profit(990, lb, y, 0, 5000, maxw, two_m) == -((y - 990) * 5000 / maxw)
    # nothing left unsettled: profit = pushed = (ub0 - lb) * D / maxW > 0
    assert O.profit(990, lb, y, 4000, 0, maxw, two_m) == (y - lb) * 4000 / maxw
    # clamping: every x <= lb - maxW has the profit of lb - maxW
    p0 = O.profit(lb - maxw, lb, y, 3000, 2000, maxw, two_m)
    assert O.profit(0, lb, y, 3000, 2000, maxw, two_m) == p0
    assert O.profit(lb - maxw - 100, lb, y, 3000, 2000, maxw, two_m) == p0
    # long edges reduce the profit relative to pushed - pulled
    p = O.profit(990, lb, y, 3000, 2000, maxw, two_m)
    assert p < (y - lb) * 3000 / maxw - (y - 990) * 2000 / maxw


# --------------------------------------------------- Algorithm 1 restatement

def _eic_cases():
    yield "urand12", G.urand(12, 15, seed=7, nsources=3)
    yield "kron12", G.kron(12, seed=31, nsources=3)
    yield "kron14_lognormal", G.kron(14, seed=32, weights="lognormal", nsources=2)
    yield "grid64", G.road(64, seed=33, wmax=4095, nsources=2)
    w = G.kron(11, seed=34, nsources=2)
    w.w = np.ones_like(w.w)  # one distinct weight: many equal-length paths
    yield "kron11_unit", w


@pytest.mark.parametrize("name,wl", list(_eic_cases()))
def test_eic_restatement_exact(name, wl):
    g = O.Graph(wl.n, wl.src, wl.dst, wl.w)
    for s in wl.sources:
        d, rc = g.dijkstra(int(s))
        de, rc2, trace, tot = g.eic(int(s))
        assert rc == rc2 == 0
        assert (de == d).all(), name
        _check_trace_against_exact(g, d, trace, tot)


def _check_trace_against_exact(g, d, trace, tot):
    assert tot["st0"] == trace[0]["ub"]
    check_trace_against_exact(g, d, trace)


def test_eic_random_small_graphs_exact():
    rng = random.Random(21)
    for trial in range(120):
        n = rng.randrange(2, 80)
        wv = rng.choice([[1], [1, 2], [1, 2, 3], list(range(1, 256)), [5, 1000, 60000]])
        src, dst, w = _rand_tuples(rng, n, rng.randrange(0, 5 * n), wv)
        g = O.Graph(n, src, dst, w)
        s = rng.randrange(n)
        d, _ = g.dijkstra(s)
        de, rc, trace, tot = g.eic(s)
        assert rc == 0 and (de == d).all(), trial
        if g.nnz:
            _check_trace_against_exact(g, d, trace, tot)


def test_eic_paper_bands_on_kron():
    """Section 4.3/4.4 bands: nFrontier ~1, nTrav ~3-5 per reachable vertex."""
    bands = _golden("bands.txt")
    wl = G.kron(15, seed=2, nsources=2)
    g = O.Graph(wl.n, wl.src, wl.dst, wl.w)
    for s in wl.sources:
        d, _ = g.dijkstra(int(s))
        _, _, _, tot = g.eic(int(s))
        reach = int((d != O.INF).sum())
        assert tot["frontier"] / reach <= bands["nfrontier_max"]
        assert bands["ntrav_min"] <= tot["traversed"] / reach <= bands["ntrav_max"]
        assert tot["traversed"] < g.m  # fewer traversals than Dijkstra's |E| (Section 4.4)


def test_oracle_traces_equal_the_golden_file():
    """The oracle's Algorithm 1 step traces on the fixture workloads equal the
    stored ones (golden/eic_traces.txt, written by golden/make_golden.py): any
    change to the oracle's arithmetic shows up here and must come with a
    regenerated file."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    with open(os.path.join(GOLDEN, "eic_traces.txt")) as f:
        want = [tuple(line.split()) for line in f if line.strip() and not line.startswith("#")]
    got = [tuple(str(v) for v in row) for row in mg.traces()]
    assert len(want) > 40
    assert got == want


def test_wide_weight_cases_reach_function2_profit():
    """The GPU parity cases with weights of 2^20 and above (where Function 2
    sums D(x') from the settled list) do evaluate Function 2's profits: some
    step's st is a grid candidate, neither lb nor lb - maxW (Section 3.2)."""
    for wmax, scale, seed in ((1 << 21, 12, 90), (1 << 24, 12, 90), (1 << 27, 13, 91)):
        wl = G.kron(scale, seed=seed, weights=f"uniform:{wmax}", nsources=3)
        g = O.Graph(wl.n, wl.src, wl.dst, wl.w)
        assert g.maxw >= 1 << 20
        for s in wl.sources:
            d, rc = g.dijkstra(int(s))
            de, rc2, trace, tot = g.eic(int(s))
            assert rc == rc2 == 0 and (de == d).all()
            assert any(r["st"] not in (r["lb"], r["lb"] - g.maxw) for r in trace[1:]), (wmax, int(s))
            _check_trace_against_exact(g, d, trace, tot)
