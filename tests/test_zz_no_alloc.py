"""eic_sssp_noalloc: the allocation-free query entry point (GPU).

Some callers cannot allocate device memory while they serve queries (a fixed
device-memory budget planned up front, another framework's memory pool, or a
latency-critical loop that cannot take cudaMalloc's implicit synchronisation).
For them libeic offers eic_sssp_noalloc, which runs the same query with a
fixed scratch array inside the library. These tests call it through the C ABI
and require, on two calls in a row, the same distances as eic_sssp and as the
oracle's Dijkstra; a clear error for a graph above each of its limits; and a
usable scratch after a query that ran out of steps. The file is named to be
collected last.
"""
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


def _noalloc(g, s, dist):
    lib = binding.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    return lib.eic_sssp_noalloc(g.handle, int(s), dist.data_ptr(), stream)


@pytest.mark.parametrize("wl", [G.kron(14, seed=50, nsources=2), G.road(96, seed=51, wmax=4095, nsources=2),
                                G.urand(13, 16, seed=52, nsources=2)], ids=["kron14", "grid96", "urand13"])
def test_noalloc_matches_eic_sssp_and_dijkstra_on_two_calls(wl):
    g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    og = O.Graph(wl.n, wl.src, wl.dst, wl.w)
    out = torch.empty(wl.n, dtype=torch.int32, device="cuda")
    for s in wl.sources[:2]:  # two calls in a row share the library's scratch
        want, orc = og.dijkstra(int(s))
        assert orc == 0
        ref, rc, _ = eic.sssp(g, int(s))
        out.fill_(7)
        assert _noalloc(g, s, out) == binding.OK
        got = eic.to_host_u32(out)
        assert np.array_equal(got, eic.to_host_u32(ref))
        assert np.array_equal(got, want)


def test_noalloc_rejects_graphs_above_each_limit():
    # more vertices than EIC_NOALLOC_MAX_VERTICES
    n = binding.NOALLOC_MAX_VERTICES + 1
    src = np.arange(0, 100, dtype=np.uint32)
    g = eic.Graph(n, src, src + 1, np.ones(100, np.uint32))
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    assert _noalloc(g, 0, out) == binding.ESIZE
    assert _noalloc(g, n, out) == binding.EINVAL
    # a weight above EIC_NOALLOC_MAX_WEIGHT
    w = np.ones(100, np.uint32)
    w[37] = binding.NOALLOC_MAX_WEIGHT + 1
    g = eic.Graph(128, src, src + 1, w)
    out = torch.empty(128, dtype=torch.int32, device="cuda")
    assert _noalloc(g, 0, out) == binding.ESIZE
    # more directed entries than EIC_NOALLOC_MAX_ENTRIES within the vertex limit
    wl = G.kron(18, seed=53, nsources=1)
    g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    assert wl.n <= binding.NOALLOC_MAX_VERTICES and 2 * g.m > binding.NOALLOC_MAX_ENTRIES
    out = torch.empty(wl.n, dtype=torch.int32, device="cuda")
    assert _noalloc(g, int(wl.sources[0]), out) == binding.ESIZE


def test_noalloc_step_limit_then_next_call_exact():
    # a 40000-vertex path takes more than EIC_NOALLOC_MAX_STEPS steps (Eq. 3 gives
    # maxW(G, 1) on a path, so each step advances about 255 distance units)
    n = 40000
    src = np.arange(n - 1, dtype=np.uint32)
    w = (src * 7 % 255 + 1).astype(np.uint32)
    g = eic.Graph(n, src, src + 1, w)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    assert _noalloc(g, 0, out) == binding.ENOMEM
    d, rc, info = eic.sssp(g, 0, stats=True)
    assert rc == 0 and info["steps"] > binding.NOALLOC_MAX_STEPS
    assert np.array_equal(eic.to_host_u32(d), np.concatenate([[0], np.cumsum(w)]).astype(np.uint32))
    # the scratch serves the next call in full
    wl = G.kron(12, seed=54, nsources=1)
    g2 = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    out2 = torch.empty(wl.n, dtype=torch.int32, device="cuda")
    assert _noalloc(g2, int(wl.sources[0]), out2) == binding.OK
    want, _ = O.Graph(wl.n, wl.src, wl.dst, wl.w).dijkstra(int(wl.sources[0]))
    assert np.array_equal(eic.to_host_u32(out2), want)
