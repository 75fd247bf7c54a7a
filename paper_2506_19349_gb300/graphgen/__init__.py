"""Seeded synthetic graph inputs for the EIC shortest-path workloads.

This module produces edge lists, weights and source vertices only; it holds
none of the shortest-path arithmetic. The generators live in ``graphgen.c``
(counter-based SplitMix64, so any thread count gives identical output) and are
loaded through ctypes. Both the CUDA path and the CPU oracle consume these
inputs.

Workload recipes (``make``) mirror the shapes of the paper's evaluation graphs
(Section 4.2, Table 1): a uniform random graph (Urand), an RMAT/Kronecker graph
(Kron, Graph500 parameters a,b,c,d = 0.57,0.19,0.19,0.05, edge factor 16), a
perturbed 4-neighbour grid standing in for Road, and a heavy-tailed log-normal
weight variant of the Kronecker topology (the paper's weight variants, Eq. 7-8,
change the weight distribution of a fixed topology).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u32p = ctypes.c_void_p
            lib.gg_rand.restype = ctypes.c_uint64
            lib.gg_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_uniform.restype = ctypes.c_int
            lib.gg_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.gg_permutation.restype = ctypes.c_int
            lib.gg_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
            lib.gg_rmat.restype = ctypes.c_int
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, u32p, u32p, ctypes.c_int]
            lib.gg_grid.restype = ctypes.c_int
            lib.gg_grid.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, u32p, u32p,
                                    ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
            lib.gg_weights_uniform.restype = None
            lib.gg_weights_uniform.argtypes = [ctypes.c_uint64, u32p, u32p, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint32, u32p, ctypes.c_int]
            lib.gg_weights_discretize.restype = None
            lib.gg_weights_discretize.argtypes = [ctypes.c_uint64, u32p, u32p, ctypes.c_uint64, ctypes.c_uint32,
                                                  u32p, ctypes.c_int]
            lib.gg_weights_converge.restype = None
            lib.gg_weights_converge.argtypes = [ctypes.c_uint64, u32p, u32p, ctypes.c_uint64, ctypes.c_double,
                                                u32p, ctypes.c_int]
            lib.gg_discretize_value.restype = ctypes.c_uint32
            lib.gg_discretize_value.argtypes = [ctypes.c_double, ctypes.c_uint32]
            lib.gg_converge_value.restype = ctypes.c_double
            lib.gg_converge_value.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.gg_weights_lognormal.restype = None
            lib.gg_weights_lognormal.argtypes = [ctypes.c_uint64, u32p, u32p, ctypes.c_uint64, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, u32p,
                                                 ctypes.c_int]
            lib.gg_pick_sources.restype = ctypes.c_int64
            lib.gg_pick_sources.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, ctypes.c_uint32,
                                            ctypes.c_uint64, ctypes.c_int, u32p]
            _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _ptr(a: np.ndarray) -> int:
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data


def _out(n: int, out) -> np.ndarray:
    if out is None:
        return np.empty(n, dtype=np.uint32)
    assert out.dtype == np.uint32 and out.size >= n
    return out[:n]


def rand(seed: int, stream: int, i: int) -> int:
    """Draw i of stream ``stream`` under ``seed`` (SplitMix64 output)."""
    return int(_load().gg_rand(seed, stream, i))


def uniform(n: int, m: int, seed: int):
    """Exactly m distinct undirected pairs, endpoints uniform in [0, n)."""
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    if _load().gg_uniform(n, m, seed, _ptr(src), _ptr(dst)) != 0:
        raise ValueError("uniform graph: m not achievable")
    return src, dst


def permutation(n: int, seed: int) -> np.ndarray:
    p = np.empty(n, dtype=np.uint32)
    _load().gg_permutation(n, seed, _ptr(p))
    return p


def rmat(scale: int, nedges: int, seed: int, a=0.57, b=0.19, c=0.19, permute=True, out_src=None, out_dst=None):
    """nedges raw RMAT tuples on 2^scale vertices (loops/duplicates kept)."""
    src = _out(nedges, out_src)
    dst = _out(nedges, out_dst)
    if _load().gg_rmat(scale, nedges, a, b, c, seed, 1 if permute else 0, _ptr(src), _ptr(dst), _threads()) != 0:
        raise ValueError("rmat: bad scale")
    return src, dst


def grid(side: int, p_del: float, diag_frac: float, seed: int):
    """side x side 4-neighbour grid with deletions and diagonal shortcuts."""
    ne = 2 * side * (side - 1)
    cap = ne + int(round(diag_frac * ne)) + 16
    src = np.empty(cap, dtype=np.uint32)
    dst = np.empty(cap, dtype=np.uint32)
    cnt = ctypes.c_uint64(0)
    if _load().gg_grid(side, p_del, diag_frac, seed, _ptr(src), _ptr(dst), cap, ctypes.byref(cnt)) != 0:
        raise ValueError("grid: capacity")
    k = int(cnt.value)
    return src[:k].copy(), dst[:k].copy()


def weights_uniform(src, dst, seed: int, wmin: int, wmax: int, out=None) -> np.ndarray:
    w = _out(src.size, out)
    _load().gg_weights_uniform(src.size, _ptr(src), _ptr(dst), seed, wmin, wmax, _ptr(w), _threads())
    return w


def weights_discretize(src, dst, seed: int, power: int, out=None) -> np.ndarray:
    """The paper's power variant (Eq. 7): 1 + round(x (2^power - 2)), x uniform in (0,1] per pair."""
    if not 1 <= power <= 31:
        raise ValueError("power must be in 1..31")
    w = out if out is not None else np.empty(src.size, dtype=np.uint32)
    _load().gg_weights_discretize(src.size, _ptr(src), _ptr(dst), seed, power, _ptr(w), _threads())
    return w


def weights_converge(src, dst, seed: int, pivot: float, out=None) -> np.ndarray:
    """The paper's pivot variant (Eq. 8), quantised to 1..65535 by Eq. 7 with power 16."""
    if not 0.0 < pivot < 1.0:
        raise ValueError("pivot must be in (0, 1)")
    w = out if out is not None else np.empty(src.size, dtype=np.uint32)
    _load().gg_weights_converge(src.size, _ptr(src), _ptr(dst), seed, pivot, _ptr(w), _threads())
    return w


def discretize(x: float, power: int) -> int:
    """Eq. 7 on one value, rounded to the nearest integer (halves up)."""
    return int(_load().gg_discretize_value(x, power))


def converge(x: float, pivot: float) -> float:
    """Eq. 8 on one value."""
    return float(_load().gg_converge_value(x, pivot))


def weights_lognormal(src, dst, seed: int, mu: float, sigma: float, wmin: int, wmax: int, out=None) -> np.ndarray:
    w = _out(src.size, out)
    _load().gg_weights_lognormal(src.size, _ptr(src), _ptr(dst), seed, mu, sigma, wmin, wmax, _ptr(w), _threads())
    return w


def pick_sources(n: int, src, dst, count: int, seed: int, mode: str = "nonisolated") -> np.ndarray:
    """count sources uniform over non-isolated vertices or the largest component."""
    out = np.empty(count, dtype=np.uint32)
    pool = _load().gg_pick_sources(n, src.size, _ptr(src), _ptr(dst), count, seed,
                                   0 if mode == "nonisolated" else 1, _ptr(out))
    if pool <= 0:
        raise ValueError("no eligible source vertex")
    return out


@dataclass
class Workload:
    """One synthetic graph: raw tuples (may hold loops/duplicates) + sources."""
    name: str
    n: int
    src: np.ndarray
    dst: np.ndarray
    w: np.ndarray
    sources: np.ndarray
    recipe: str
    meta: dict = field(default_factory=dict)

    @property
    def num_tuples(self) -> int:
        return int(self.src.size)


def kron(scale: int, seed: int = 2, edgefactor: int = 16, weights: str = "uniform255", nsources: int = 64,
         source_seed: int | None = None, out=None) -> Workload:
    """RMAT scale/edgefactor graph, ids permuted, weights per unordered pair.

    weights: "uniform255" -> integers uniform in [1,255];
             "uniform:W"  -> integers uniform in [1,W];
             "lognormal"  -> clamp(llround(exp(3 + 1.5 Z)), 1, 65535);
             "power:P"    -> the paper's power variant, Eq. 7 with power P;
             "pivot:Y"    -> the paper's pivot variant, Eq. 8 with pivot Y, as integers 1..65535.
    Sources: uniform over vertices with at least one non-loop edge.
    """
    ne = edgefactor << scale
    o = out or {}
    src, dst = rmat(scale, ne, seed, out_src=o.get("src"), out_dst=o.get("dst"))
    if weights == "uniform255":
        w = weights_uniform(src, dst, seed, 1, 255, out=o.get("w"))
    elif weights.startswith("uniform:"):
        w = weights_uniform(src, dst, seed, 1, int(weights[8:]), out=o.get("w"))
    elif weights == "lognormal":
        w = weights_lognormal(src, dst, seed, 3.0, 1.5, 1, 65535, out=o.get("w"))
    elif weights.startswith("power:"):
        w = weights_discretize(src, dst, seed, int(weights[6:]), out=o.get("w"))
    elif weights.startswith("pivot:"):
        w = weights_converge(src, dst, seed, float(weights[6:]), out=o.get("w"))
    else:
        raise ValueError(weights)
    ss = seed if source_seed is None else source_seed
    srcs = pick_sources(1 << scale, src, dst, nsources, ss, "nonisolated")
    return Workload(f"kron{scale}" + ("" if weights == "uniform255" else "_" + weights), 1 << scale, src, dst, w,
                    srcs, f"RMAT(0.57,0.19,0.19,0.05) scale {scale} edgefactor {edgefactor} seed {seed}, "
                          f"permuted ids, weights {weights}", {"scale": scale, "seed": seed})


def urand(log_n: int = 14, log_m: int = 17, seed: int = 1, nsources: int = 1) -> Workload:
    n, m = 1 << log_n, 1 << log_m
    src, dst = uniform(n, m, seed)
    w = weights_uniform(src, dst, seed, 1, 255)
    srcs = pick_sources(n, src, dst, nsources, seed, "largest")
    return Workload(f"urand{log_n}", n, src, dst, w, srcs,
                    f"uniform random: n=2^{log_n}, exactly 2^{log_m} distinct undirected edges, seed {seed}, "
                    f"weights uniform [1,255]", {"log_n": log_n})


def road(side: int = 4096, seed: int = 3, wmax: int = 4095, nsources: int = 16) -> Workload:
    src, dst = grid(side, 0.10, 0.02, seed)
    w = weights_uniform(src, dst, seed, 1, wmax)
    srcs = pick_sources(side * side, src, dst, nsources, seed, "largest")
    return Workload(f"grid{side}", side * side, src, dst, w, srcs,
                    f"{side}x{side} grid, 10% of 4-neighbour edges deleted, 2% diagonal shortcuts, seed {seed}, "
                    f"weights uniform [1,{wmax}]", {"side": side})


def batch_set(kron_scales=range(12, 23), grid_sides=((256, 3), (512, 3), (1024, 2), (2048, 2)),
              nsources: int = 8) -> list[Workload]:
    """32 graphs of uneven size: Kron scales 12..22 twice (seeds 40+s, 60+s)
    and grids 256^2 x3, 512^2 x3, 1024^2 x2, 2048^2 x2, weights in [1,255]."""
    out = []
    for s in kron_scales:
        for base in (40, 60):
            out.append(kron(s, seed=base + s, nsources=nsources))
    gi = 0
    for side, reps in grid_sides:
        for r in range(reps):
            out.append(road(side, seed=100 + gi, wmax=255, nsources=nsources))
            gi += 1
    return out
