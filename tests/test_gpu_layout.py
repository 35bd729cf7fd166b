"""Per-graph layouts (the SpMV's row split: chunk length of long rows and the
sliced-ELL row limit) and the layout autotuner.  Every layout changes only the
order of floating-point sums: each must match the float64 oracle at the
mixed-precision tolerance (1e-6 per quantity), for narrow and wide walks."""
import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth

pytestmark = pytest.mark.gpu

LAYOUTS = [(32, 8), (256, 32), (512, 64), (4096, 64), (65536, 16)]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08143_gb300 import fj
    c = fj.Context(0)
    yield c
    c.set_layout()
    c.close()


@pytest.fixture(scope="module")
def problem():
    g = synth.chung_lu(60_000, 300_000, 2.1, seed=121, weighted=True)
    s = synth.opinions_batch_mix(g.n, 16, 122)
    z = fo.solve(g.n, g.src, g.dst, g.w, s).reshape(g.n, -1)
    q = [fo.quantities_from_z(g.n, g.src, g.dst, g.w, s[:, j], z[:, j]) for j in range(s.shape[1])]
    return g, s, z, q


def _check(q, qo, s):
    for name in fo.QUANTITY_NAMES:
        assert fo.relative_error(qo[name], q[name], 1e-12 * float(s @ s)) <= 1e-6, name


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("k", [1, 16])
def test_every_layout_matches_the_oracle(ctx, problem, layout, k):
    g, s, zo, qo = problem
    ctx.set_layout(*layout)
    try:
        with ctx.upload_edges(g) as dg:
            assert dg.layout() == {"chunk_len": layout[0], "sell_max": layout[1]}
            z, q, info = ctx.solve(dg, s[:, :k])
    finally:
        ctx.set_layout()
    assert info["rel_residual"] <= 1e-10
    for j in range(k):
        _check(q[j], qo[j], s[:, j])
    np.testing.assert_allclose(z, zo[:, :k], rtol=0, atol=1e-8)


def test_weight_update_under_a_small_sliced_ell_limit(ctx, problem):
    """A weight update on a graph whose sliced ELL holds rows of at most 8
    entries (most rows are chunked) is the same bits as a fresh upload."""
    g, s, _, _ = problem
    rng = np.random.default_rng(5)
    idx = rng.choice(g.m, 3000, replace=False)
    w2 = g.w.copy()
    w2[idx] = (1.0 - rng.random(idx.shape[0])).astype(np.float32)
    g2 = synth.EdgeList(g.n, g.src, g.dst, w2)
    ctx.set_layout(128, 8)
    try:
        with ctx.upload_edges(g) as dg, ctx.upload_edges(g2) as fresh:
            dg.update_weights(g.src[idx], g.dst[idx], w2[idx])
            z1, q1, _ = ctx.solve(dg, s[:, :2])
            z2, q2, _ = ctx.solve(fresh, s[:, :2])
    finally:
        ctx.set_layout()
    assert np.array_equal(z1, z2) and q1 == q2


def test_layout_tuner_picks_and_applies_a_layout(ctx, problem):
    from paper_2101_08143_gb300 import fj
    g, s, _, qo = problem
    try:
        res = ctx.tune_layout(g.n, g.src, g.dst, g.w, s[:, 0], repeats=2)
        assert res["best"] in res["ms"] and len(res["ms"]) >= 8
        assert (512, 64) in res["ms"]
        assert res["ms"][res["best"]] == min(res["ms"].values())
        with ctx.upload_edges(g) as dg:
            assert (dg.layout()["chunk_len"], dg.layout()["sell_max"]) == res["best"]
            _, q, _ = ctx.solve(dg, s[:, 0])
        _check(q[0], qo[0], s[:, 0])
    finally:
        ctx.set_layout()
    lib = fj.load()
    bad = fj.Layout(16, 64)
    assert lib.fj_set_layout(ctx.handle, bad) == fj.FJ_ERR_ARG
    bad = fj.Layout(512, 65)
    assert lib.fj_set_layout(ctx.handle, bad) == fj.FJ_ERR_ARG
