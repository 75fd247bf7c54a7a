"""CPU oracle for the EIC shortest-path method — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never imports, links or executes it, and it shares no code with
that path. The arithmetic lives in ``oracle.c`` (plain C, fp64 built with
``-ffp-contract=off``); this module compiles it with gcc and wraps it with
ctypes.

Functions and the passages of the paper (arXiv 2506.19349) they follow:
  - ``Graph``: CSR built by the oracle itself from raw tuples (symmetrised,
    self-loops dropped, duplicate pairs keep the minimum weight, rows sorted by
    (weight, neighbour): the per-vertex weight order of Section 4.1).
  - ``Graph.dijkstra``: dist[v] = lsp(s, v), the problem definition of
    Section 2, by binary-heap Dijkstra (pinned against Bellman-Ford,
    Floyd-Warshall, closed forms and the invariant checker).
  - ``bellman_ford`` / ``floyd_warshall``: the classical algorithms of
    Section 2.2 on the raw tuple list (tiny inputs).
  - ``Graph.check``: invariant certificate of a distance array
    (``check_many``: the same over several arrays on host threads).
  - ``rtow``: maxW(G, ratio) quantile table RtoW (Section 3, Section 4.1).
  - ``highd``: highD over a degree multiset (Section 3).
  - ``gap``: Eq. 1-3. ``profit``: Eq. 4-6 with the clamping of Section 3.2.
  - ``Graph.eic``: sequential Algorithm 1 with Function 1 and Function 2,
    returning distances, the per-step trace and the counters of Section 4.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

INF = 0xFFFFFFFF
INF_T = 1 << 62

ALPHA, BETA, RATIO_NUM, ST_NUM = 3, 0.9, 4096, 1024  # Section 4.1 settings


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Step(ctypes.Structure):
    _fields_ = [("lb", ctypes.c_int64), ("ub", ctypes.c_int64), ("st", ctypes.c_int64), ("gap_lb", ctypes.c_int64),
                ("sumd_lb", ctypes.c_uint64), ("highd_lb", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("settled", ctypes.c_uint64), ("push_set", ctypes.c_uint64), ("pull_set", ctypes.c_uint64),
                ("push_trav", ctypes.c_uint64), ("pull_trav", ctypes.c_uint64), ("frontier", ctypes.c_uint64),
                ("improved", ctypes.c_uint64)]


class _Totals(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("rounds", ctypes.c_uint64), ("frontier", ctypes.c_uint64),
                ("traversed", ctypes.c_uint64), ("push_trav", ctypes.c_uint64), ("pull_trav", ctypes.c_uint64),
                ("improved", ctypes.c_uint64), ("st0", ctypes.c_int64), ("st1", ctypes.c_int64)]


class _Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_uint32), ("beta", ctypes.c_double), ("ratio_num", ctypes.c_uint32),
                ("st_num", ctypes.c_uint32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            vp, u32, u64, i64, dbl = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_double
            L.og_build.restype = vp
            L.og_build.argtypes = [u32, u64, vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            L.og_free.argtypes = [vp]
            L.og_free.restype = None
            for name, rt in (("og_n", u32), ("og_nnz", u64), ("og_maxw", u32), ("og_maxdeg", u32)):
                getattr(L, name).restype = rt
                getattr(L, name).argtypes = [vp]
            L.og_export.argtypes = [vp, vp, vp, vp]
            L.og_export.restype = None
            L.og_dijkstra.argtypes = [vp, u32, vp]
            L.og_dijkstra.restype = ctypes.c_int
            L.og_dijkstra_many.argtypes = [vp, u32, vp, vp, vp, ctypes.c_int]
            L.og_dijkstra_many.restype = None
            L.og_bellman_ford.argtypes = [u32, u64, vp, vp, vp, u32, vp]
            L.og_bellman_ford.restype = ctypes.c_int
            L.og_floyd_warshall.argtypes = [u32, u64, vp, vp, vp, u32, vp]
            L.og_floyd_warshall.restype = ctypes.c_int
            L.og_check.argtypes = [vp, u32, vp, ctypes.POINTER(ctypes.c_uint32)]
            L.og_check.restype = ctypes.c_int
            L.og_parent.argtypes = [vp, u32, vp, vp]
            L.og_parent.restype = None
            L.og_rtow_from_weights.argtypes = [u64, vp, u32, vp]
            L.og_rtow_from_weights.restype = ctypes.c_int
            L.og_rtow.argtypes = [vp, u32, vp]
            L.og_rtow.restype = ctypes.c_int
            L.og_highd_list.argtypes = [u64, vp]
            L.og_highd_list.restype = u64
            L.og_gap.argtypes = [u64, u64, u64, u32, dbl, u32, vp, ctypes.POINTER(ctypes.c_uint32),
                                 ctypes.POINTER(ctypes.c_double)]
            L.og_gap.restype = i64
            L.og_profit.argtypes = [i64, i64, i64, u64, u64, u32, u64]
            L.og_profit.restype = dbl
            L.og_eic.argtypes = [vp, u32, ctypes.POINTER(_Params), vp, ctypes.POINTER(_Step), u64,
                                 ctypes.POINTER(_Totals)]
            L.og_eic.restype = ctypes.c_int
            L.og_stats_at.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
            L.og_stats_at.restype = None
            L.og_degree_between.argtypes = [vp, vp, i64, i64]
            L.og_degree_between.restype = u64
            _lib = L
    return _lib


def _u32(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a


class OracleError(RuntimeError):
    pass


class Graph:
    """Undirected CSR built by the oracle from raw (src, dst, w) tuples."""

    def __init__(self, n: int, src, dst, w, nthreads: int | None = None):
        L = _load()
        self._keep = (_u32(src), _u32(dst), _u32(w))
        s, d, ww = self._keep
        if not (s.size == d.size == ww.size):
            raise ValueError("tuple arrays differ in length")
        err = ctypes.c_int(0)
        nt = nthreads or max(1, min(32, os.cpu_count() or 1))
        self._h = L.og_build(n, s.size, s.ctypes.data, d.ctypes.data, ww.ctypes.data, nt, ctypes.byref(err))
        self._keep = None
        if not self._h:
            raise OracleError({1: "invalid tuple (endpoint >= n or weight 0)", 2: "out of memory"}.get(err.value,
                                                                                                       "error"))
        self.n = int(L.og_n(self._h))
        self.nnz = int(L.og_nnz(self._h))
        self.m = self.nnz // 2
        self.maxw = int(L.og_maxw(self._h))
        self.maxdeg = int(L.og_maxdeg(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.og_free(h)
            self._h = None

    def csr(self):
        row = np.empty(self.n + 1, dtype=np.uint64)
        nbr = np.empty(self.nnz, dtype=np.uint32)
        w = np.empty(self.nnz, dtype=np.uint32)
        _load().og_export(self._h, row.ctypes.data, nbr.ctypes.data, w.ctypes.data)
        return row, nbr, w

    def degrees(self) -> np.ndarray:
        row, _, _ = self.csr()
        return np.diff(row).astype(np.uint64)

    def dijkstra(self, s: int) -> np.ndarray:
        """(dist, rc): rc 0 ok, 3 overflow (max lsp + maxW >= 2^32-1)."""
        dist = np.empty(self.n, dtype=np.uint32)
        rc = _load().og_dijkstra(self._h, int(s), dist.ctypes.data)
        if rc in (1, 2):
            raise OracleError(f"dijkstra rc={rc}")
        return dist, rc

    def dijkstra_many(self, sources, nthreads: int | None = None):
        srcs = _u32(sources)
        k = srcs.size
        dists = np.empty((k, self.n), dtype=np.uint32)
        rcs = np.zeros(k, dtype=np.int32)
        nt = nthreads or max(1, min(k, os.cpu_count() or 1))
        _load().og_dijkstra_many(self._h, k, srcs.ctypes.data, dists.ctypes.data, rcs.ctypes.data, nt)
        return dists, rcs

    def check(self, s: int, dist) -> tuple[int, int]:
        """(code, vertex): 0 ok; 1 dist[s]!=0; 2 violated edge; 3 no tight edge; 4 reachability."""
        d = _u32(dist)
        bad = ctypes.c_uint32(0)
        rc = _load().og_check(self._h, int(s), d.ctypes.data, ctypes.byref(bad))
        return int(rc), int(bad.value)

    def check_many(self, sources, dists, nthreads: int | None = None) -> list[tuple[int, int]]:
        """check() of each (sources[i], dists[i]) on host threads (the C call
        releases the interpreter lock, so the checks run in parallel)."""
        from concurrent.futures import ThreadPoolExecutor

        pairs = list(zip(sources, dists))
        nt = max(1, min(len(pairs), nthreads or os.cpu_count() or 1))
        with ThreadPoolExecutor(nt) as ex:
            return list(ex.map(lambda p: self.check(int(p[0]), p[1]), pairs))

    def parent(self, s: int, dist) -> np.ndarray:
        d = _u32(dist)
        p = np.empty(self.n, dtype=np.uint32)
        _load().og_parent(self._h, int(s), d.ctypes.data, p.ctypes.data)
        return p

    def rtow(self, R: int = RATIO_NUM) -> np.ndarray:
        out = np.empty(R, dtype=np.uint32)
        if _load().og_rtow(self._h, R, out.ctypes.data) != 0:
            raise OracleError("rtow")
        return out

    def stats_at(self, dist, x: int) -> tuple[int, int]:
        """(sumD(x), highD(x)) over {v : dist[v] >= x} of a final distance array."""
        d = _u32(dist)
        sd, hd = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _load().og_stats_at(self._h, d.ctypes.data, int(x), ctypes.byref(sd), ctypes.byref(hd))
        return int(sd.value), int(hd.value)

    def degree_between(self, dist, x: int, y: int) -> int:
        d = _u32(dist)
        return int(_load().og_degree_between(self._h, d.ctypes.data, int(x), int(y)))

    def eic(self, s: int, alpha=ALPHA, beta=BETA, ratio_num=RATIO_NUM, st_num=ST_NUM, trace_cap: int = 1 << 20):
        """Sequential Algorithm 1: (dist, rc, trace: list[dict], totals: dict)."""
        dist = np.empty(self.n, dtype=np.uint32)
        prm = _Params(alpha, beta, ratio_num, st_num)
        cap = max(1, min(trace_cap, 1 << 20))
        tr = (_Step * cap)()
        tot = _Totals()
        rc = _load().og_eic(self._h, int(s), ctypes.byref(prm), dist.ctypes.data, tr, cap, ctypes.byref(tot))
        if rc in (1, 2):
            raise OracleError(f"eic rc={rc}")
        nsteps = int(tot.steps)
        trace = [{f: getattr(tr[i], f) for f, _ in _Step._fields_} for i in range(min(nsteps, cap))]
        totals = {f: getattr(tot, f) for f, _ in _Totals._fields_}
        return dist, rc, trace, totals


def bellman_ford(n: int, src, dst, w, s: int) -> tuple[np.ndarray, int]:
    s_, d_, w_ = _u32(src), _u32(dst), _u32(w)
    dist = np.empty(n, dtype=np.uint32)
    rc = _load().og_bellman_ford(n, s_.size, s_.ctypes.data, d_.ctypes.data, w_.ctypes.data, int(s), dist.ctypes.data)
    return dist, rc


def floyd_warshall(n: int, src, dst, w, s: int) -> np.ndarray:
    s_, d_, w_ = _u32(src), _u32(dst), _u32(w)
    dist = np.empty(n, dtype=np.uint32)
    rc = _load().og_floyd_warshall(n, s_.size, s_.ctypes.data, d_.ctypes.data, w_.ctypes.data, int(s),
                                   dist.ctypes.data)
    if rc:
        raise OracleError(f"floyd_warshall rc={rc}")
    return dist


def rtow(weights, R: int = RATIO_NUM) -> np.ndarray:
    """RtoW[i] = maxW(G, i/(R-1)) over an undirected weight multiset."""
    ws = _u32(weights)
    out = np.empty(R, dtype=np.uint32)
    if _load().og_rtow_from_weights(ws.size, ws.ctypes.data, R, out.ctypes.data) != 0:
        raise OracleError("rtow: empty weight set")
    return out


def highd(degrees) -> int:
    d = _u32(degrees)
    return int(_load().og_highd_list(d.size, d.ctypes.data))


def gap(sumd: int, highd_: int, two_m: int, rtow_table, alpha=ALPHA, beta=BETA) -> tuple[int, int, float]:
    """(gap, RtoW index, ratio) by Eq. 1-3."""
    t = _u32(rtow_table)
    idx, ratio = ctypes.c_uint32(0), ctypes.c_double(0)
    g = _load().og_gap(sumd, highd_, two_m, alpha, beta, t.size, t.ctypes.data, ctypes.byref(idx),
                       ctypes.byref(ratio))
    return int(g), int(idx.value), float(ratio.value)


def profit(x: int, lb: int, y: int, dsum: int, sumd_lb: int, maxw: int, two_m: int) -> float:
    """Eq. 4-6 profit with the Section 3.2 clamping (dsum = sumD(x') - sumD(lb))."""
    return float(_load().og_profit(x, lb, y, dsum, sumd_lb, maxw, two_m))
