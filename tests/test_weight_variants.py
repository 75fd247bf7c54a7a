"""The paper's weight variants (Section 4.2, Eq. 7-8) as input generators, and
the oracle's Algorithm 1 staying exact on them (no GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2506_19349_gb300 import graphgen as G


@pytest.mark.parametrize("power", [1, 2, 3, 8, 10, 16])
def test_discretize_maps_onto_the_integers_1_to_2p_minus_1(power):
    top = (1 << power) - 1
    assert G.discretize(1.0, power) == top
    assert G.discretize(2.0 ** -60, power) == 1
    if power > 1:  # rounding: the first step up is at x = 1/2 of a unit
        unit = 1.0 / ((1 << power) - 2)
        assert G.discretize(0.49 * unit, power) == 1 and G.discretize(0.51 * unit, power) == 2
    xs = np.linspace(1e-9, 1.0, 4001)
    vals = [G.discretize(float(x), power) for x in xs]
    assert all(a <= b for a, b in zip(vals, vals[1:]))  # monotone
    assert min(vals) >= 1 and max(vals) == top
    # x = k / (2^p - 2) lands exactly on 1 + k (Eq. 7 without rounding error at the knots)
    if power > 1:
        for k in range(0, (1 << power) - 1, max(1, (1 << power) // 16)):
            assert G.discretize(k / ((1 << power) - 2), power) == 1 + k


def test_discretize_weights_cover_every_value():
    wl = G.kron(12, seed=7, weights="power:3", nsources=1)
    assert set(np.unique(wl.w).tolist()) == set(range(1, 8))
    wl = G.kron(10, seed=7, weights="power:1", nsources=1)
    assert (wl.w == 1).all()  # 2^1 - 2 = 0: every weight is 1


@pytest.mark.parametrize("pivot", [0.1, 0.3, 0.5, 0.9])
def test_converge_shape(pivot):
    assert G.converge(0.5, pivot) == pytest.approx(pivot, abs=0)
    assert G.converge(1.0, pivot) == pytest.approx(1.0)
    assert G.converge(1e-15, pivot) == pytest.approx(0.0, abs=1e-12)
    xs = np.linspace(1e-9, 1.0, 2001)
    vals = [G.converge(float(x), pivot) for x in xs]
    assert all(a <= b + 1e-15 for a, b in zip(vals, vals[1:]))  # monotone
    # the two branches: y - y(1-2x)^2 below one half, y + (1-y)(1-2x)^2 above
    assert G.converge(0.25, pivot) == pytest.approx(pivot - pivot * 0.25)
    assert G.converge(0.75, pivot) == pytest.approx(pivot + (1 - pivot) * 0.25)


@pytest.mark.parametrize("pivot", [0.2, 0.7])
def test_pivot_weights_have_their_median_and_peak_at_the_pivot(pivot):
    wl = G.kron(14, seed=9, weights=f"pivot:{pivot}", nsources=1)
    w = wl.w.astype(np.float64)
    assert w.min() >= 1 and w.max() <= 65535
    at_pivot = G.discretize(pivot, 16)
    assert abs(np.mean(w < at_pivot) - 0.5) < 0.02  # half of the new weights are below the pivot
    hist, edges = np.histogram(w, bins=20, range=(1, 65535))
    k = int(np.argmax(hist))  # the bell's peak: the density is unbounded at the pivot itself
    width = edges[1] - edges[0]
    assert edges[k] - width <= at_pivot <= edges[k + 1] + width


def test_variant_weights_are_functions_of_the_pair():
    wl = G.kron(10, seed=11, weights="power:6", nsources=1)
    key = {}
    for u, v, w in zip(wl.src.tolist(), wl.dst.tolist(), wl.w.tolist()):
        k = (min(u, v), max(u, v))
        assert key.setdefault(k, w) == w
    again = G.kron(10, seed=11, weights="power:6", nsources=1)
    assert np.array_equal(wl.w, again.w)


@pytest.mark.parametrize("weights", ["power:1", "power:2", "power:10", "pivot:0.1", "pivot:0.9"])
def test_oracle_algorithm1_exact_on_variants(weights):
    wl = G.kron(10, seed=12, weights=weights, nsources=3)
    og = O.Graph(wl.n, wl.src, wl.dst, wl.w)
    for s in wl.sources:
        want, _ = og.dijkstra(int(s))
        got, rc, _, _ = og.eic(int(s))
        assert rc == 0 and np.array_equal(got, want)
