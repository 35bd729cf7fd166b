"""fj_graph_update_weights: new weights for existing edges of a resident
graph (the FJ model on a changed graph, Sec. 3.1), then a warm re-solve.

The updated graph must be the same bits as a fresh upload of the changed
edge list, its solve must match the float64 oracle on the changed graph
(1e-6 per quantity), and a warm start from the old equilibrium must need
fewer iterations than a cold solve.
"""
import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08143_gb300 import fj
    c = fj.Context(0)
    yield c
    c.close()


def _changed(g, frac, seed):
    rng = np.random.default_rng(seed)
    idx = rng.choice(g.m, max(1, int(frac * g.m)), replace=False)
    w_new = (1.0 - rng.random(idx.shape[0])).astype(np.float32)
    w = g.w.copy() if g.w is not None else np.ones(g.m, np.float32)
    w[idx] = w_new
    # updates name the pairs in either orientation
    flip = rng.random(idx.shape[0]) < 0.5
    su = np.where(flip, g.dst[idx], g.src[idx]).astype(np.int32)
    sv = np.where(flip, g.src[idx], g.dst[idx]).astype(np.int32)
    return synth.EdgeList(g.n, g.src, g.dst, w), su, sv, w_new


def _check(g, s, z, q):
    zo = fo.solve(g.n, g.src, g.dst, g.w, s)
    qo = fo.quantities_from_z(g.n, g.src, g.dst, g.w, s, zo)
    for name in fo.QUANTITY_NAMES:
        assert fo.relative_error(qo[name], q[name], 1e-12 * float(s @ s)) <= 1e-6, name
    np.testing.assert_allclose(z, zo, rtol=0, atol=1e-8)


@pytest.mark.parametrize("weighted", [True, False])
def test_update_then_warm_solve(ctx, weighted):
    from paper_2101_08143_gb300 import fj
    if weighted:
        g = synth.chung_lu(20_000, 100_000, 2.2, seed=91, weighted=True)
    else:
        g = synth.erdos_renyi(10_000, 50_000, seed=92)
    s = synth.opinions_uniform(g.n, 1, 93)[:, 0]
    g2, su, sv, w_new = _changed(g, 0.01, 94)
    o = fj.default_opts(tol=1e-10)
    with ctx.upload_edges(g) as dg, ctx.upload_edges(g2) as fresh:
        z1, _, _ = ctx.solve(dg, s, opts=o)
        dg.update_weights(su, sv, w_new)
        assert dg.stats() == fresh.stats()
        zc, qc, info_cold = ctx.solve(dg, s, opts=o)
        zw, qw, info_warm = ctx.solve(dg, s, opts=o, z0=z1)
        zf, qf, _ = ctx.solve(fresh, s, opts=o)
    # the updated graph is the fresh upload's bits
    assert np.array_equal(zc, zf) and qc == qf
    assert info_warm["iterations"] < info_cold["iterations"]
    _check(g2, s, zw, qw[0])


def test_update_with_device_pointers_and_hub_rows(ctx):
    """Hub rows of many chunks and rows of the sliced ELL both change."""
    import torch
    g = synth.chung_lu(60_000, 300_000, 2.1, seed=95, weighted=True)
    s = synth.opinions_uniform(g.n, 2, 96)
    g2, su, sv, w_new = _changed(g, 0.05, 97)
    with ctx.upload_edges(g) as dg, ctx.upload_edges(g2) as fresh:
        dg.update_weights(torch.from_numpy(su).cuda(), torch.from_numpy(sv).cuda(), torch.from_numpy(w_new).cuda())
        zc, qc, _ = ctx.solve(dg, s)
        zf, qf, _ = ctx.solve(fresh, s)
    assert np.array_equal(zc, zf) and qc == qf
    for j in range(2):
        _check(g2, s[:, j], zc[:, j], qc[j])


def test_bad_updates_leave_the_graph_unchanged(ctx):
    from paper_2101_08143_gb300 import fj
    g = synth.erdos_renyi(3000, 12_000, seed=98, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 99)[:, 0]
    # a pair that is not an edge
    have = set(zip(g.src.tolist(), g.dst.tolist())) | set(zip(g.dst.tolist(), g.src.tolist()))
    a, b = next((i, j) for i in range(g.n) for j in range(i + 1, g.n) if (i, j) not in have)
    with ctx.upload_edges(g) as dg:
        z0, q0, _ = ctx.solve(dg, s)
        ok_src, ok_dst = g.src[:3], g.dst[:3]
        for src, dst, w in ((np.r_[ok_src, a], np.r_[ok_dst, b], [0.5, 0.5, 0.5, 0.5]),
                            (ok_src, ok_dst, [0.5, np.nan, 0.5]),
                            (ok_src, ok_dst, [0.5, 0.0, 0.5]),
                            (np.r_[ok_src, g.n], np.r_[ok_dst, 0], [0.5, 0.5, 0.5, 0.5]),
                            (np.r_[ok_src, 7], np.r_[ok_dst, 7], [0.5, 0.5, 0.5, 0.5])):
            with pytest.raises(fj.FJError) as e:
                dg.update_weights(src, dst, np.asarray(w, np.float32))
            assert e.value.code == fj.FJ_ERR_GRAPH
        z1, q1, _ = ctx.solve(dg, s)
    assert np.array_equal(z0, z1) and q0 == q1
