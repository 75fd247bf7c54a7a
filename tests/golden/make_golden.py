"""Writes the oracle-derived fixture of this folder, ``eic_traces.txt``: the
step traces of the oracle's sequential Algorithm 1 (dynamic stepping of
Eq. 1-3, Function 1/2 with Eq. 4-6) on small seeded workloads.

It calls only ``oracle/`` and the seeded input generators, which hold none of
the method's arithmetic. Run it from the repository root:

    python tests/golden/make_golden.py

A change to the stored traces is a change to the oracle's arithmetic, and its
commit names the passage of the paper, or the reading of it, that justifies it.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "eic_traces.txt")
COLUMNS = ("lb", "ub", "st", "gap_lb", "sumd_lb", "highd_lb", "settled")


def workloads():
    """(name, workload) pairs: a uniform random graph, a Kronecker graph and a
    road-like grid, with the generators' own seeded sources."""
    sys.path.insert(0, ROOT)
    from paper_2506_19349_gb300 import graphgen as G

    return [("urand14", G.urand(14, 17, seed=1, nsources=2)),
            ("kron12", G.kron(12, seed=25, nsources=2)),
            ("grid32", G.road(32, seed=23, wmax=4095, nsources=1))]


def traces():
    """Rows (name, source, step fields...) of the oracle's Algorithm 1."""
    sys.path.insert(0, ROOT)
    import oracle as O

    rows = []
    for name, wl in workloads():
        og = O.Graph(wl.n, wl.src, wl.dst, wl.w)
        for s in wl.sources:
            _, rc, trace, _ = og.eic(int(s))
            assert rc == 0
            rows += [(name, int(s)) + tuple(int(r[c]) for c in COLUMNS) for r in trace]
    return rows


def main():
    with open(OUT, "w") as f:
        f.write("# Step traces of the oracle's sequential Algorithm 1 (oracle/oracle.c), written by\n"
                "# tests/golden/make_golden.py on the workloads it names.\n")
        f.write("# columns: workload source " + " ".join(COLUMNS) + "\n")
        for row in traces():
            f.write(" ".join(str(v) for v in row) + "\n")
    print(OUT)


if __name__ == "__main__":
    main()
