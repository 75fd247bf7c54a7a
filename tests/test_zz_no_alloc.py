"""eic_sssp_noalloc: the allocation-free query entry point (GPU).

Some callers cannot allocate device memory while they serve queries (a fixed
device-memory budget planned up front, another framework's memory pool, or a
latency-critical loop that cannot take cudaMalloc's implicit synchronisation).
For them libeic offers eic_sssp_noalloc, which runs the same query with a
fixed scratch array inside the library. These tests call it through the C ABI
and require the same distances as eic_sssp, on two calls in a row, and a clear
error for a graph above its limits. The file is named to be collected last.
"""
import numpy as np
import pytest

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
def test_noalloc_matches_eic_sssp_on_two_calls(wl):
    g = eic.Graph(wl.n, wl.src, wl.dst, wl.w)
    out = torch.empty(wl.n, dtype=torch.int32, device="cuda")
    for s in wl.sources[:2]:  # two calls in a row share the library's scratch
        want, rc, _ = eic.sssp(g, int(s))
        out.fill_(7)
        assert _noalloc(g, s, out) == binding.OK
        assert np.array_equal(eic.to_host_u32(out), eic.to_host_u32(want))


def test_noalloc_rejects_graph_above_limits():
    n = binding.NOALLOC_MAX_VERTICES + 1
    src = np.arange(0, 100, dtype=np.uint32)
    g = eic.Graph(n, src, src + 1, np.ones(100, np.uint32))
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    assert _noalloc(g, 0, out) == binding.ESIZE
    assert _noalloc(g, n, out) == binding.EINVAL
