"""The seeded generators: simple graphs, exact sizes, determinism."""
import numpy as np
import pytest

from paper_2101_08143_gb300 import synth


def _is_simple(g):
    assert np.all(g.src != g.dst)
    lo = np.minimum(g.src, g.dst).astype(np.int64)
    hi = np.maximum(g.src, g.dst).astype(np.int64)
    key = lo * g.n + hi
    assert np.unique(key).size == key.size
    assert g.src.min() >= 0 and g.dst.max() < g.n


@pytest.mark.parametrize("weighted", [False, True])
def test_erdos_renyi(weighted):
    g = synth.erdos_renyi(2000, 10000, seed=1, weighted=weighted)
    assert g.m == 10000 and g.src.dtype == np.int32
    _is_simple(g)
    if weighted:
        assert g.w.dtype == np.float32
        assert g.w.min() > 0 and g.w.max() <= 1
    else:
        assert g.w is None
    g2 = synth.erdos_renyi(2000, 10000, seed=1, weighted=weighted)
    assert np.array_equal(g.src, g2.src) and np.array_equal(g.dst, g2.dst)


def test_chung_lu_power_law_shape():
    g = synth.chung_lu(100_000, 500_000, 2.3, seed=2, weighted=True)
    assert g.m == 500_000
    _is_simple(g)
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    # heavy tail: the top node holds far more than the average degree
    assert deg.max() > 100 * deg.mean()
    # hubs are spread over the id space (ids were permuted)
    assert int(np.argmax(deg)) != 0 or deg[1:].max() < deg[0]


def test_opinions():
    s = synth.opinions_uniform(1000, 3, 5)
    assert s.shape == (1000, 3) and s.flags.f_contiguous
    assert s.min() >= 0 and s.max() < 1
    b = synth.opinions_polarized(5000, 1, 5)
    # Beta(0.5, 0.5) piles up near 0 and 1
    assert np.mean((b < 0.1) | (b > 0.9)) > 0.35
    for f in (synth.opinions_exponential, synth.opinions_power_law):
        x = f(1000, 2, 3)
        assert np.allclose(x.max(axis=0), 1.0) and x.min() > 0
    mix = synth.opinions_batch_mix(100, 8, 1)
    assert mix.shape == (100, 8)
