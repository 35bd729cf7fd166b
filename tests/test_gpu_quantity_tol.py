"""FJ_QUANTITY_TOL: the solve stops once each quantity's relative error is
certified below tol from the float64 residual.  Checked against the float64
oracle's quantities (the actual error) and against the certified bound
recomputed on the host from the oracle's residual of the GPU's z."""
import numpy as np
import pytest

import bench
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


def _oracle(g, s):
    z = fo.solve(g.n, g.src, g.dst, g.w, s, tol=1e-12)
    return z, fo.quantities_from_z(g.n, g.src, g.dst, g.w, s, z)


def _certified(g, s, z, q):
    return bench.accuracy_bound(g, s, z, q)["sigma_bound"]


@pytest.fixture(scope="module")
def bench_1m():
    spec = synth.WORKLOADS["cl_n1m_m5m_b2.3"]
    g = synth.make_graph(spec)
    s = synth.make_opinions(spec, g.n)[:, 0]
    zo, qo = _oracle(g, s)
    return g, s, zo, qo


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("tol", [1e-6, 1e-9])
def test_bench_graph_quantity_tol(ctx, bench_1m, prec, tol):
    """The 1M-node bench graph, mixed and float64 modes: every quantity
    within tol of the oracle, the certified bound within tol, and a looser
    target than residual 1e-8 takes fewer iterations."""
    import torch
    from paper_2101_08143_gb300 import fj
    g, s, zo, qo = bench_1m
    dev = torch.device("cuda")
    with ctx.upload(g.n, torch.from_numpy(g.src).to(dev), torch.from_numpy(g.dst).to(dev),
                    torch.from_numpy(g.w).to(dev), merge_duplicates=True) as dg:
        sd = torch.from_numpy(s).to(dev)
        z, q, info = ctx.solve(dg, sd, opts=fj.default_opts(tol=tol, precision=prec, flags=fj.FJ_QUANTITY_TOL))
        _, _, info_res = ctx.solve(dg, sd, opts=fj.default_opts(tol=1e-8, precision=prec))
    z = z.cpu().numpy()
    for name in fo.QUANTITY_NAMES:
        err = fo.relative_error(qo[name], q[0][name])
        assert err <= tol, (name, err)
    bound = _certified(g, s, z, q[0])
    assert max(bound.values()) <= tol, bound
    if tol >= 1e-6:
        assert info["iterations"] < info_res["iterations"], (info["iterations"], info_res["iterations"])


def test_er_graph_quantity_tol_columns(ctx):
    """Several columns, each stopped by its own certified bound (one of them
    nearly constant, so its quantities are small)."""
    from paper_2101_08143_gb300 import fj
    g = synth.erdos_renyi(5000, 30000, seed=61, weighted=True)
    S = np.asfortranarray(np.column_stack([synth.opinions_uniform(g.n, 1, 62)[:, 0],
                                           synth.opinions_polarized(g.n, 1, 63)[:, 0],
                                           0.5 + 1e-3 * synth.opinions_uniform(g.n, 1, 64)[:, 0]]))
    with ctx.upload_edges(g) as dg:
        z, q, info = ctx.solve(dg, S, opts=fj.default_opts(tol=1e-7, flags=fj.FJ_QUANTITY_TOL))
    for j in range(S.shape[1]):
        _, qo = _oracle(g, S[:, j])
        for name in fo.QUANTITY_NAMES:
            assert fo.relative_error(qo[name], q[j][name]) <= 1e-7, (j, name)
        assert max(_certified(g, S[:, j], z[:, j], q[j]).values()) <= 1e-7


def test_quantity_tol_batch_and_served(ctx):
    """The flag reaches packed batches and served requests: both meet the
    target, and a batch part is the same bits as the own solve on its grid."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(20000, 80000, 2.3, seed=65, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 66)
    o = fj.default_opts(tol=1e-6, flags=fj.FJ_QUANTITY_TOL)
    _, qo = _oracle(g, s[:, 0])
    with ctx.upload_edges(g) as dg:
        rc, parts = ctx.solve_batch([dg, dg], [s, s], opts=o)
        assert rc == fj.FJ_OK
        ctx.set_grid(parts[0][2]["blocks"])
        try:
            _, q_own, _ = ctx.solve(dg, s, opts=o)
        finally:
            ctx.set_grid(0)
    for z, q, info in parts:
        assert q[0] == q_own[0]
        for name in fo.QUANTITY_NAMES:
            assert fo.relative_error(qo[name], q[0][name]) <= 1e-6
    rc, q_srv, info = fj.poll(ctx, fj.submit_edges(ctx, g.n, g.src, g.dst, g.w, s, opts=o), -1)
    assert rc == fj.FJ_OK
    for name in fo.QUANTITY_NAMES:
        assert fo.relative_error(qo[name], q_srv[0][name]) <= 1e-6


def test_quantity_tol_rejected_where_undefined(ctx):
    from paper_2101_08143_gb300 import fj
    g = synth.erdos_renyi(100, 300, seed=67)
    s = synth.opinions_uniform(g.n, 1, 68)
    with ctx.upload_edges(g) as dg:
        for o in (fj.default_opts(tol=1e-6, precision=fj.PREC_FP32, flags=fj.FJ_QUANTITY_TOL),
                  fj.default_opts(tol=1e-6, flags=fj.FJ_QUANTITY_TOL | fj.FJ_TWO_SOLVES)):
            with pytest.raises(fj.FJError) as e:
                ctx.solve(dg, s, opts=o)
            assert e.value.code == fj.FJ_ERR_ARG


def test_quantity_tol_degenerate_inputs(ctx):
    """Edgeless graph (L = 0, z = s, D = 0 bounds nothing), constant opinions
    (s_bar = 0), and 33 columns (launches of 32 and 1), all with the rule."""
    from paper_2101_08143_gb300 import fj
    o = fj.default_opts(tol=1e-6, flags=fj.FJ_QUANTITY_TOL)
    g = synth.edgeless(1000)
    s = synth.opinions_uniform(g.n, 1, 70)
    with ctx.upload_edges(g) as dg:
        z, q, info = ctx.solve(dg, s, opts=o)
    np.testing.assert_allclose(z[:, 0] if z.ndim == 2 else z, s[:, 0], atol=1e-12)
    _, qo = _oracle(g, s[:, 0])
    for name in fo.QUANTITY_NAMES:
        assert fo.relative_error(qo[name], q[0][name], floor=1e-12) <= 1e-6, name
    g = synth.chung_lu(3000, 12000, 2.3, seed=71, weighted=True)
    with ctx.upload_edges(g) as dg:
        sc = np.full((g.n, 1), 0.25)
        z, q, info = ctx.solve(dg, sc, opts=o)
        np.testing.assert_allclose(z[:, 0] if z.ndim == 2 else z, 0.25, atol=1e-14)
        assert q[0]["C_I"] == 0.0 and q[0]["D"] == 0.0 and q[0]["P"] == 0.0
        S = synth.opinions_uniform(g.n, 33, 72)
        z, q, info = ctx.solve(dg, S, opts=o)
    for j in (0, 31, 32):
        _, qo = _oracle(g, S[:, j])
        for name in fo.QUANTITY_NAMES:
            assert fo.relative_error(qo[name], q[j][name]) <= 1e-6, (j, name)


def test_quantity_tol_warm_start(ctx):
    """fj_solve_warm under the rule: from the solution of nearby opinions it
    needs fewer iterations and still meets the target."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(50_000, 250_000, 2.2, seed=73, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 74)[:, 0]
    s2 = s.copy()
    idx = np.random.default_rng(75).choice(g.n, g.n // 100, replace=False)
    s2[idx] += np.random.default_rng(76).uniform(-0.01, 0.01, len(idx))
    o = fj.default_opts(tol=1e-6, flags=fj.FJ_QUANTITY_TOL)
    _, qo = _oracle(g, s2)
    with ctx.upload_edges(g) as dg:
        z1, _, _ = ctx.solve(dg, s, opts=o)
        _, q_cold, i_cold = ctx.solve(dg, s2, opts=o)
        _, q_warm, i_warm = ctx.solve(dg, s2, opts=o, z0=z1)
    assert i_warm["iterations"] < i_cold["iterations"]
    for q in (q_cold, q_warm):
        for name in fo.QUANTITY_NAMES:
            assert fo.relative_error(qo[name], q[0][name]) <= 1e-6, name
