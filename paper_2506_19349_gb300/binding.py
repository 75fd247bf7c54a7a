"""Thin ctypes binding over libeic (include/eic.h). Argument marshalling only.

Every step of a query runs in libeic's CUDA kernels; this module passes
pointers and sizes. PyTorch supplies device memory and streams. There is no
CPU fallback: loading fails loudly when the library or a CUDA device is
missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeic.so")

EIC_INF = 0xFFFFFFFF
RATIO_NUM = 4096
OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, ETIMEOUT, EBUSY, ESIZE, EABORT = range(9)
NOALLOC_MAX_VERTICES = 1 << 18  # the EIC_NOALLOC_* limits of include/eic.h
NOALLOC_MAX_ENTRIES = 1 << 22
NOALLOC_MAX_WEIGHT = 65535
NOALLOC_MAX_DEGREES = 4096
NOALLOC_MAX_STEPS = 1 << 14
FLAG_NO_PULL = 1
FLAG_NO_FUSE = 2

# Every name declared in include/eic.h.
EXPORTS = ("eic_params_default", "eic_strerror", "eic_version", "eic_graph_create", "eic_graph_info",
           "eic_graph_export", "eic_graph_export_internal", "eic_graph_memory", "eic_graph_destroy", "eic_sssp", "eic_sssp_batch",
           "eic_sssp_noalloc", "eic_batch_create", "eic_batch_run", "eic_batch_wait", "eic_batch_tune",
           "eic_batch_info", "eic_batch_gap_shifts", "eic_batch_destroy", "eic_server_create", "eic_server_submit", "eic_server_poll",
           "eic_server_wait", "eic_server_result", "eic_server_release", "eic_server_stats",
           "eic_server_reset_stats", "eic_server_tune", "eic_server_destroy")


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_uint32), ("beta", ctypes.c_double), ("st_num", ctypes.c_uint32),
                ("gap_shift", ctypes.c_uint32), ("block_threads", ctypes.c_uint32), ("heavy_min", ctypes.c_uint32),
                ("max_spin_log2", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("batch_groups", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 7)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_uint32), ("blocks_per_group", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("cuda_graph", ctypes.c_uint32), ("gap_shift", ctypes.c_uint32), ("heavy_min", ctypes.c_uint32),
                ("queries", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("scratch_bytes", ctypes.c_uint64),
                ("tuned_ms", ctypes.c_double)]


class Step(ctypes.Structure):
    _fields_ = [("lb", ctypes.c_int64), ("ub", ctypes.c_int64), ("st", ctypes.c_int64), ("gap_lb", ctypes.c_int64),
                ("sumd_lb", ctypes.c_uint64), ("highd_lb", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("settled", ctypes.c_uint64), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


STEP_PULL = 1   # EIC_STEP_PULL: Function 1's pull ran in the step (st < lb)
STEP_SWEPT = 2  # EIC_STEP_SWEPT: the pull went over the unsettled vertices in vertex order


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("rounds", ctypes.c_uint64), ("frontier", ctypes.c_uint64),
                ("traversed", ctypes.c_uint64), ("pulls", ctypes.c_uint64), ("improved", ctypes.c_uint64),
                ("heavy", ctypes.c_uint64), ("pull_items", ctypes.c_uint64), ("trace", ctypes.POINTER(Step)),
                ("trace_cap", ctypes.c_uint64),
                ("trace_len", ctypes.c_uint64), ("timeline", ctypes.POINTER(ctypes.c_uint64)),
                ("timeline_cap", ctypes.c_uint64), ("timeline_len", ctypes.c_uint64), ("kernel_ms", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_uint32), ("ring_entries", ctypes.c_uint32), ("output_bytes", ctypes.c_uint64),
                ("idle_us", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 5)]


class ServerReport(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "admitted", "completed", "queued", "in_flight",
                                               "max_in_flight", "kernel_launches", "output_bytes_used",
                                               "output_bytes", "scratch_bytes")] + \
               [("groups", ctypes.c_uint32), ("blocks_per_group", ctypes.c_uint32),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_mean_ms", ctypes.c_double), ("latency_count", ctypes.c_uint64)]


class EicError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else f"{strerror(status)} ({status})")


_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Load libeic.so (raises if it is absent: no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libeic.so not found at {p}: build it first (paper_2506_19349_gb300.build)")
        L = ctypes.CDLL(p)
        vp, u32, u64, c_int = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        L.eic_params_default.argtypes = [ctypes.POINTER(Params)]
        L.eic_params_default.restype = c_int
        L.eic_strerror.argtypes = [c_int]
        L.eic_strerror.restype = ctypes.c_char_p
        L.eic_version.argtypes = []
        L.eic_version.restype = c_int
        L.eic_graph_create.argtypes = [vp, vp, vp, u64, u32, c_int, vp, ctypes.POINTER(vp)]
        L.eic_graph_create.restype = c_int
        L.eic_graph_info.argtypes = [vp] + [ctypes.POINTER(u32), ctypes.POINTER(u64)] + [ctypes.POINTER(u32)] * 4
        L.eic_graph_info.restype = c_int
        L.eic_graph_export.argtypes = [vp, vp, vp, vp, vp]
        L.eic_graph_export.restype = c_int
        L.eic_graph_export_internal.argtypes = [vp, ctypes.POINTER(u32), vp, vp, vp, vp]
        L.eic_graph_export_internal.restype = c_int
        L.eic_graph_memory.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.eic_graph_memory.restype = c_int
        L.eic_graph_destroy.argtypes = [vp]
        L.eic_graph_destroy.restype = c_int
        L.eic_sssp.argtypes = [vp, u32, vp, vp, ctypes.POINTER(Params), ctypes.POINTER(Stats), vp]
        L.eic_sssp.restype = c_int
        L.eic_sssp_batch.argtypes = [ctypes.POINTER(vp), vp, u32, ctypes.POINTER(vp), ctypes.POINTER(Params), vp, vp]
        L.eic_sssp_batch.restype = c_int
        L.eic_sssp_noalloc.argtypes = [vp, u32, vp, vp]
        L.eic_sssp_noalloc.restype = c_int
        L.eic_batch_create.argtypes = [ctypes.POINTER(vp), vp, u32, ctypes.POINTER(vp), ctypes.POINTER(Params),
                                       ctypes.POINTER(vp)]
        L.eic_batch_create.restype = c_int
        L.eic_batch_run.argtypes = [vp, vp]
        L.eic_batch_run.restype = c_int
        L.eic_batch_wait.argtypes = [vp, vp, vp]
        L.eic_batch_wait.restype = c_int
        L.eic_batch_tune.argtypes = [vp, vp, ctypes.POINTER(BatchConfig)]
        L.eic_batch_tune.restype = c_int
        L.eic_batch_info.argtypes = [vp, ctypes.POINTER(BatchConfig)]
        L.eic_batch_info.restype = c_int
        L.eic_batch_gap_shifts.argtypes = [vp, vp]
        L.eic_batch_gap_shifts.restype = c_int
        L.eic_batch_destroy.argtypes = [vp]
        L.eic_batch_destroy.restype = c_int
        L.eic_server_create.argtypes = [ctypes.POINTER(vp), u32, ctypes.POINTER(Params), ctypes.POINTER(ServerConfig),
                                        ctypes.POINTER(vp)]
        L.eic_server_create.restype = c_int
        L.eic_server_submit.argtypes = [vp, u32, u32, ctypes.POINTER(u64)]
        L.eic_server_submit.restype = c_int
        L.eic_server_poll.argtypes = [vp, u64, ctypes.POINTER(c_int)]
        L.eic_server_poll.restype = c_int
        L.eic_server_wait.argtypes = [vp, u64, u32, ctypes.POINTER(c_int)]
        L.eic_server_wait.restype = c_int
        L.eic_server_result.argtypes = [vp, u64, vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double)]
        L.eic_server_result.restype = c_int
        L.eic_server_release.argtypes = [vp, u64]
        L.eic_server_release.restype = c_int
        L.eic_server_stats.argtypes = [vp, ctypes.POINTER(ServerReport)]
        L.eic_server_stats.restype = c_int
        L.eic_server_reset_stats.argtypes = [vp]
        L.eic_server_reset_stats.restype = c_int
        L.eic_server_tune.argtypes = [vp, vp, vp]
        L.eic_server_tune.restype = c_int
        L.eic_server_destroy.argtypes = [vp]
        L.eic_server_destroy.restype = c_int
        _lib = L
        return L


def strerror(status: int) -> str:
    try:
        return load_library().eic_strerror(status).decode()
    except Exception:  # pragma: no cover - only when the library cannot load
        return f"status {status}"


def default_params(**overrides) -> Params:
    p = Params()
    load_library().eic_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("libeic needs a CUDA device")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check(status: int, what: str):
    if status != OK:
        raise EicError(status, what)


class Graph:
    """Device-resident graph (eic_graph_create / eic_graph_destroy)."""

    def __init__(self, n: int, src, dst, w, stream=None):
        torch = _torch()
        L = load_library()
        self._h = ctypes.c_void_p()
        keep = []
        if isinstance(src, torch.Tensor) and src.is_cuda:
            t = [x.contiguous() for x in (src, dst, w)]
            assert all(x.dtype in (torch.int32, torch.uint32) for x in t)
            keep = t
            ptrs = [x.data_ptr() for x in t]
            num, on_dev = t[0].numel(), 1
        else:
            a = [np.ascontiguousarray(x, dtype=np.uint32) for x in (src, dst, w)]
            keep = a
            ptrs = [x.ctypes.data for x in a]
            num, on_dev = a[0].size, 0
        st = _stream_ptr(stream)
        rc = L.eic_graph_create(ptrs[0], ptrs[1], ptrs[2], num, n, on_dev, st, ctypes.byref(self._h))
        del keep
        _check(rc, "eic_graph_create")
        nn, m, md, mw, mi, h0 = (ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32(),
                                 ctypes.c_uint32(), ctypes.c_uint32())
        _check(L.eic_graph_info(self._h, ctypes.byref(nn), ctypes.byref(m), ctypes.byref(md), ctypes.byref(mw),
                                ctypes.byref(mi), ctypes.byref(h0)), "eic_graph_info")
        self.n, self.m, self.max_deg, self.max_w, self.min_w, self.highd0 = (nn.value, m.value, md.value, mw.value,
                                                                            mi.value, h0.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.eic_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self):
        """(row_ptr uint64[n+1], nbr uint32[2m], w uint32[2m], rtow uint32[4096]) on the host."""
        row = np.empty(self.n + 1, dtype=np.uint64)
        nbr = np.empty(2 * self.m, dtype=np.uint32)
        w = np.empty(2 * self.m, dtype=np.uint32)
        rt = np.empty(RATIO_NUM, dtype=np.uint32)
        _check(load_library().eic_graph_export(self._h, row.ctypes.data, nbr.ctypes.data, w.ctypes.data,
                                               rt.ctypes.data), "eic_graph_export")
        return row, nbr, w, rt

    def export_internal(self):
        """The CSR in the device's internal order: (int2orig uint32[ni], row
        uint32[ni+1], nbr uint32[2m] internal ids, w uint32[2m])."""
        L = load_library()
        ni = ctypes.c_uint32()
        _check(L.eic_graph_export_internal(self._h, ctypes.byref(ni), None, None, None, None),
               "eic_graph_export_internal")
        i2o = np.empty(ni.value, dtype=np.uint32)
        row = np.empty(ni.value + 1, dtype=np.uint32)
        nbr = np.empty(2 * self.m, dtype=np.uint32)
        w = np.empty(2 * self.m, dtype=np.uint32)
        _check(L.eic_graph_export_internal(self._h, ctypes.byref(ni), i2o.ctypes.data, row.ctypes.data,
                                           nbr.ctypes.data, w.ctypes.data), "eic_graph_export_internal")
        return i2o, row, nbr, w

    def memory(self):
        gb, wb = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load_library().eic_graph_memory(self._h, ctypes.byref(gb), ctypes.byref(wb)), "eic_graph_memory")
        return gb.value, wb.value


def new_dist(n: int, device=None):
    torch = _torch()
    return torch.empty(n, dtype=torch.int32, device=device or "cuda")


def sssp(graph: Graph, source: int, dist=None, parent=None, params: Params | None = None, stats: bool = False,
         trace_cap: int = 0, stream=None, raise_on_error: bool = True, timeline_cap: int = 0):
    """One query. Returns (dist, status, stats_dict or None); dist is an int32
    CUDA tensor holding uint32 distances (0xFFFFFFFF = unreachable)."""
    L = load_library()
    if dist is None:
        dist = new_dist(graph.n)
    st = Stats()
    rows = None
    if trace_cap:
        rows = (Step * trace_cap)()
        st.trace = ctypes.cast(rows, ctypes.POINTER(Step))
        st.trace_cap = trace_cap
    tl = None
    if timeline_cap:
        tl = np.zeros(2 * timeline_cap, dtype=np.uint64)
        st.timeline = tl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        st.timeline_cap = timeline_cap
    want = stats or trace_cap or timeline_cap
    rc = L.eic_sssp(graph.handle, int(source), dist.data_ptr(), parent.data_ptr() if parent is not None else None,
                    ctypes.byref(params) if params is not None else None, ctypes.byref(st) if want else None,
                    _stream_ptr(stream))
    if raise_on_error:
        _check(rc, "eic_sssp")
    info = None
    if want:
        info = {f: getattr(st, f) for f, _ in Stats._fields_ if f not in ("trace", "trace_cap", "timeline",
                                                                           "timeline_cap")}
        if tl is not None:
            k = min(st.timeline_len, timeline_cap)
            info["timeline"] = tl[:2 * k].reshape(k, 2)
        if rows is not None:
            info["trace"] = [{f: getattr(rows[i], f) for f, _ in Step._fields_}
                             for i in range(min(st.trace_len, trace_cap))]
    return dist, rc, info


def sssp_batch(graphs, sources, dists, params: Params | None = None, stream=None):
    """Queries (graphs[i], sources[i]) -> dists[i] (CUDA tensors); returns the statuses."""
    L = load_library()
    q = len(sources)
    harr = (ctypes.c_void_p * q)(*[g.handle.value for g in graphs])
    srcs = np.ascontiguousarray(sources, dtype=np.uint32)
    darr = (ctypes.c_void_p * q)(*[d.data_ptr() for d in dists])
    statuses = np.zeros(q, dtype=np.int32)
    L.eic_sssp_batch(harr, srcs.ctypes.data, q, darr, ctypes.byref(params) if params is not None else None,
                     statuses.ctypes.data, _stream_ptr(stream))
    return statuses


def _config_dict(c: BatchConfig) -> dict:
    return {f: getattr(c, f) for f, _ in BatchConfig._fields_ if f != "reserved"}


class Batch:
    """A prepared batch (eic_batch_*): queries (graphs[i], sources[i]) ->
    dists[i] in one persistent launch, replayed as a CUDA graph."""

    def __init__(self, graphs, sources, dists, params: Params | None = None):
        L = load_library()
        self._graphs = list(graphs)  # keep the graphs and outputs alive with the batch
        self.dists = list(dists)
        q = len(sources)
        harr = (ctypes.c_void_p * q)(*[g.handle.value for g in self._graphs])
        self._srcs = np.ascontiguousarray(sources, dtype=np.uint32)
        darr = (ctypes.c_void_p * q)(*[d.data_ptr() for d in self.dists])
        self._h = ctypes.c_void_p()
        _check(L.eic_batch_create(harr, self._srcs.ctypes.data, q, darr,
                                  ctypes.byref(params) if params is not None else None, ctypes.byref(self._h)),
               "eic_batch_create")
        self.n = q

    def run(self, stream=None):
        _check(load_library().eic_batch_run(self._h, _stream_ptr(stream)), "eic_batch_run")

    def wait(self, stream=None) -> np.ndarray:
        st = np.zeros(self.n, dtype=np.int32)
        load_library().eic_batch_wait(self._h, _stream_ptr(stream), st.ctypes.data)
        return st

    def tune(self, stream=None) -> dict:
        c = BatchConfig()
        _check(load_library().eic_batch_tune(self._h, _stream_ptr(stream), ctypes.byref(c)), "eic_batch_tune")
        return _config_dict(c)

    def info(self) -> dict:
        c = BatchConfig()
        _check(load_library().eic_batch_info(self._h, ctypes.byref(c)), "eic_batch_info")
        return _config_dict(c)

    def gap_shifts(self) -> list:
        """Each query's step-width scaling in use (the tuner picks it per graph)."""
        out = np.zeros(self.n, dtype=np.uint32)
        _check(load_library().eic_batch_gap_shifts(self._h, out.ctypes.data), "eic_batch_gap_shifts")
        return out.tolist()

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.eic_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over resident graphs (eic_server_*)."""

    def __init__(self, graphs, params: Params | None = None, groups: int = 0, ring_entries: int = 0,
                 output_bytes: int = 0, idle_us: int = 0):
        L = load_library()
        self._graphs = list(graphs)  # the server reads them until it is closed
        harr = (ctypes.c_void_p * len(self._graphs))(*[g.handle.value for g in self._graphs])
        cfg = ServerConfig(groups=groups, ring_entries=ring_entries, output_bytes=output_bytes, idle_us=idle_us)
        self._h = ctypes.c_void_p()
        _check(L.eic_server_create(harr, len(self._graphs), ctypes.byref(params) if params is not None else None,
                                   ctypes.byref(cfg), ctypes.byref(self._h)), "eic_server_create")

    def submit(self, graph: int, source: int) -> int:
        t = ctypes.c_uint64()
        _check(load_library().eic_server_submit(self._h, graph, source, ctypes.byref(t)), "eic_server_submit")
        return t.value

    def poll(self, ticket: int):
        """Status once done, else None."""
        st = ctypes.c_int()
        rc = load_library().eic_server_poll(self._h, ticket, ctypes.byref(st))
        if rc == EBUSY:
            return None
        _check(rc, "eic_server_poll")
        return st.value

    def wait(self, ticket: int, timeout_ms: int = 60000) -> int:
        st = ctypes.c_int()
        _check(load_library().eic_server_wait(self._h, ticket, timeout_ms, ctypes.byref(st)), "eic_server_wait")
        return st.value

    def result(self, ticket: int, n: int | None = None, to_host: bool = True):
        """(distances as a host uint32 array or None, latency in ms) of a done request."""
        lat = ctypes.c_double()
        if to_host:
            if n is None:
                raise ValueError("n is required to copy the result to the host")
            out = np.empty(n, dtype=np.uint32)
            _check(load_library().eic_server_result(self._h, ticket, out.ctypes.data, None, ctypes.byref(lat)),
                   "eic_server_result")
            return out, lat.value
        _check(load_library().eic_server_result(self._h, ticket, None, None, ctypes.byref(lat)), "eic_server_result")
        return None, lat.value

    def release(self, ticket: int):
        _check(load_library().eic_server_release(self._h, ticket), "eic_server_release")

    def stats(self) -> dict:
        r = ServerReport()
        _check(load_library().eic_server_stats(self._h, ctypes.byref(r)), "eic_server_stats")
        return {f: getattr(r, f) for f, _ in ServerReport._fields_}

    def reset_stats(self):
        _check(load_library().eic_server_reset_stats(self._h), "eic_server_reset_stats")

    def tune(self, sample_sources) -> list:
        """Per resident graph, the step-width scaling that serves its sample
        source fastest (eic_server_tune); returns the chosen values."""
        src = np.ascontiguousarray(sample_sources, dtype=np.uint32)
        if src.size != len(self._graphs):
            raise ValueError("one sample source per resident graph")
        out = np.zeros(src.size, dtype=np.uint32)
        _check(load_library().eic_server_tune(self._h, src.ctypes.data, out.ctypes.data), "eic_server_tune")
        return out.tolist()

    def close(self):
        if getattr(self, "_h", None) and self._h.value and _lib is not None:
            _lib.eic_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def to_host_u32(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def sssp_noalloc(graph: Graph, source: int, dist, stream=None) -> int:
    """eic_sssp_noalloc: the query with libeic's fixed scratch instead of the
    graph's workspace, for callers that cannot allocate device memory at query
    time. dist is a caller-provided int32 CUDA tensor of n elements. Returns the
    status code."""
    return load_library().eic_sssp_noalloc(graph.handle, int(source), dist.data_ptr(), _stream_ptr(stream))
