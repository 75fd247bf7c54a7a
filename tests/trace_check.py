"""A step trace of Algorithm 1 checked against the exact distances (test helper).

Every quantity of a step boundary is a function of the exact shortest
distances (Section 3): sumD and highD over VS(lb) = {dist >= lb}, the gap of
Eq. 1-3, the vertices settled in [lb, ub), the first step's final ub (the
smallest distance among the vertices of degree >= highD(0)), the termination
rule of Algorithm 1, and st by Function 2 over the ST_NUM grid of Section 4.1
with the clamped estimates of Eq. 4-6. Only the oracle's functions are used.
"""
import oracle as O


def check_trace_against_exact(g, d, trace):
    """g: oracle.Graph; d: exact distances (uint32, caller's ids); trace: rows
    with lb, ub, st, gap_lb, sumd_lb, highd_lb, settled."""
    rt = g.rtow()
    deg = g.degrees()
    highd0 = O.highd(deg)
    fin = d != O.INF
    hi = deg >= highd0
    st0 = int(d[hi & fin].min()) if (hi & fin).any() else O.INF_T
    assert trace[0]["lb"] == 0 and trace[0]["ub"] == st0
    for k, row in enumerate(trace):
        sumd, highd = g.stats_at(d, row["lb"])
        assert (row["sumd_lb"], row["highd_lb"]) == (sumd, highd), k
        assert row["gap_lb"] == O.gap(sumd, highd, g.nnz, rt)[0], k
        if k > 0:
            assert row["lb"] == trace[k - 1]["ub"]
            assert row["ub"] == row["lb"] + row["gap_lb"]
        if row["ub"] < O.INF_T:
            assert row["settled"] == int(((d >= row["lb"]) & (d < row["ub"]) & fin).sum()), k
    # termination rule of Algorithm 1: the first boundary with max lsp + maxW < lb
    mx = int(d[fin].max())
    assert mx + g.maxw < trace[-1]["ub"]
    for row in trace[:-1]:
        assert mx + g.maxw >= row["ub"]
    # Function 2 at each boundary, from exact distances
    m = g.nnz // 2
    st1 = next((r["lb"] for r in trace[1:] if r["sumd_lb"] <= m), None)
    cache = {}
    for k in range(1, len(trace)):
        ub, sumd_ub = trace[k]["lb"], trace[k]["sumd_lb"]
        gap_lb, gap_ub = trace[k - 1]["gap_lb"], trace[k]["gap_lb"]
        if sumd_ub >= m or gap_lb == g.maxw:
            want = ub
        elif gap_ub == g.maxw:
            want = ub - g.maxw
        else:
            y = ub + gap_ub
            want, best = ub, 0.0
            for j in range(O.ST_NUM + 1):
                x = st0 + (j * (st1 - st0)) // O.ST_NUM
                if x >= ub:
                    continue
                xc = max(x, ub - g.maxw)
                if (xc, ub) not in cache:
                    cache[(xc, ub)] = g.degree_between(d, xc, ub)
                p = O.profit(x, ub, y, cache[(xc, ub)], sumd_ub, g.maxw, g.nnz)
                if best < p:
                    best, want = p, x
        assert trace[k]["st"] == want, k
