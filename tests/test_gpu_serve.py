"""GPU parity of the serving path: requests admitted while others are in
flight give exactly the oracle's (and eic_sssp's) distances, alone and in
the mix; admission respects the result-memory budget; the kernel is
relaunched after going idle; errors stay with their request."""
import time

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


@pytest.fixture(scope="module")
def resident():
    wls = [G.kron(11, seed=120, nsources=1), G.kron(13, seed=121, nsources=1),
           G.road(64, seed=122, wmax=255, nsources=1), G.urand(12, 14, seed=123, nsources=1)]
    graphs = [eic.Graph(w.n, w.src, w.dst, w.w) for w in wls]
    oracles = [O.Graph(w.n, w.src, w.dst, w.w) for w in wls]
    return graphs, oracles


class _Want:
    def __init__(self, graphs, oracles):
        self.graphs, self.oracles, self.cache = graphs, oracles, {}

    def __call__(self, gi, s):
        if (gi, s) not in self.cache:
            self.cache[(gi, s)] = self.oracles[gi].dijkstra(s)[0]
        return self.cache[(gi, s)]


def test_served_results_equal_alone_and_in_the_mix(resident):
    graphs, oracles = resident
    want = _Want(graphs, oracles)
    rng = np.random.default_rng(5)
    reqs = [(int(g), int(rng.integers(graphs[g].n))) for g in rng.integers(0, len(graphs), 120)]
    reqs += reqs[:10]  # repeated requests
    srv = eic.Server(graphs, groups=8)
    tickets = [srv.submit(g, s) for g, s in reqs]
    for t, (g, s) in zip(tickets, reqs):
        assert srv.wait(t) == 0
        got, lat = srv.result(t, graphs[g].n)
        assert lat > 0
        assert np.array_equal(got, want(g, s)), (g, s)
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["in_flight"] == 0 and st["queued"] == 0
    assert st["latency_count"] == len(reqs) and st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
    srv.close()
    # alone: the plain path gives the same bytes
    for g, s in reqs[:12]:
        d, rc, _ = eic.sssp(graphs[g], s)
        assert np.array_equal(eic.to_host_u32(d), want(g, s))


def test_poisson_arrivals_and_relaunch_after_idle(resident):
    graphs, oracles = resident
    want = _Want(graphs, oracles)
    rng = np.random.default_rng(6)
    srv = eic.Server(graphs, groups=4, idle_us=300)
    done = []
    for burst in range(2):
        tickets = []
        for _ in range(25):
            g = int(rng.integers(len(graphs)))
            s = int(rng.integers(graphs[g].n))
            tickets.append((srv.submit(g, s), g, s))
            time.sleep(float(rng.exponential(0.002)))  # Poisson stream, 500 req/s
        for t, g, s in tickets:
            assert srv.wait(t) == 0
            got, _ = srv.result(t, graphs[g].n)
            assert np.array_equal(got, want(g, s))
            srv.release(t)
            done.append(t)
        time.sleep(0.3)  # longer than every idle bound: the kernel leaves
    st = srv.stats()
    assert st["completed"] == 50
    assert st["kernel_launches"] >= 2
    srv.close()


def test_admission_keeps_results_within_the_memory_budget(resident):
    graphs, oracles = resident
    want = _Want(graphs, oracles)
    g = 1
    n = graphs[g].n
    budget = 2 * ((4 * n + 255) // 256) * 256  # room for two results
    srv = eic.Server(graphs, groups=4, output_bytes=budget)
    srcs = [int(x) for x in np.random.default_rng(7).integers(n, size=12)]
    tickets = [srv.submit(g, s) for s in srcs]
    time.sleep(0.05)
    st = srv.stats()
    assert st["admitted"] <= 2 and st["queued"] >= 10  # the rest waits for memory
    for t, s in zip(tickets, srcs):
        assert srv.wait(t) == 0
        got, _ = srv.result(t, n)
        assert np.array_equal(got, want(g, s))
        srv.release(t)  # frees room for the next one
    st = srv.stats()
    assert st["completed"] == 12 and st["max_in_flight"] <= 2 and st["output_bytes_used"] == 0
    with pytest.raises(eic.EicError) as e:
        small = eic.Server(graphs, output_bytes=1024)
        small.submit(g, 0)
    assert e.value.status == binding.ENOMEM
    srv.close()


def test_errors_stay_with_their_request(resident):
    graphs, oracles = resident
    want = _Want(graphs, oracles)
    n = 300
    a = np.arange(n - 1, dtype=np.uint32)
    bad = eic.Graph(n, a, a + 1, np.full(n - 1, 100_000_000, np.uint32))  # distances overflow
    srv = eic.Server([graphs[0], bad], groups=2)
    with pytest.raises(eic.EicError):
        srv.submit(2, 0)  # no such graph
    with pytest.raises(eic.EicError):
        srv.submit(0, graphs[0].n)  # no such vertex
    tb = srv.submit(1, 0)
    good = [(srv.submit(0, s), s) for s in range(0, 40, 4)]
    assert srv.wait(tb) == binding.EOVERFLOW
    for t, s in good:
        assert srv.wait(t) == 0
        got, _ = srv.result(t, graphs[0].n)
        assert np.array_equal(got, want(0, s))
        srv.release(t)
    # the failed request's group may have stopped; later requests still run
    t2 = srv.submit(0, 5)
    assert srv.wait(t2) == 0
    srv.release(t2)
    srv.release(tb)
    srv.close()


def test_destroy_with_requests_pending(resident):
    graphs, _ = resident
    srv = eic.Server(graphs, groups=2)
    for k in range(60):
        srv.submit(k % len(graphs), 0)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30


def test_tuned_server_stays_exact(resident):
    graphs, oracles = resident
    want = _Want(graphs, oracles)
    srv = eic.Server(graphs, groups=4)
    shifts = srv.tune([0] * len(graphs))
    assert len(shifts) == len(graphs) and all(0 <= x <= 8 for x in shifts)
    rng = np.random.default_rng(8)
    reqs = [(int(g), int(rng.integers(graphs[g].n))) for g in rng.integers(0, len(graphs), 40)]
    tickets = [srv.submit(g, s) for g, s in reqs]
    for t, (g, s) in zip(tickets, reqs):
        assert srv.wait(t) == 0
        got, _ = srv.result(t, graphs[g].n)
        assert np.array_equal(got, want(g, s)), (g, s)
        srv.release(t)
    # tuning needs an idle server
    t = srv.submit(0, 1)
    try:
        srv.tune([0] * len(graphs))
    except eic.EicError as e:
        assert e.status == binding.EBUSY
    srv.wait(t)
    srv.release(t)
    srv.close()
