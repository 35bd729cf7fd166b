"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative error per quantity, the paper's sigma = |rho - rho~|/rho):
  mixed (float32 inner + float64 refinement) and float64 modes: 1e-6
  pure float32 mode: 1e-3
"""
import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-6, 1: 1e-6, 2: 1e-3}  # by precision mode


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08143_gb300 import fj
    c = fj.Context(0)
    yield c
    c.close()


def _floor(s):
    return 1e-12 * float(np.sum(np.asarray(s) ** 2))


def _check_quantities(gq, oq, s, rtol):
    for name in fo.QUANTITY_NAMES:
        err = fo.relative_error(oq[name], gq[name], floor=_floor(s))
        assert err <= rtol, (name, gq[name], oq[name], err)


def _oracle_edges(n, src, dst, w, s, tol=1e-12):
    s = np.asarray(s, dtype=np.float64).reshape(n, -1)
    z = fo.solve(n, src, dst, w, s, tol=tol).reshape(n, -1)
    q = [fo.quantities_from_z(n, src, dst, w, s[:, j], z[:, j]) for j in range(s.shape[1])]
    return z, q


def _oracle(g, s, tol=1e-12):
    s = np.asarray(s, dtype=np.float64).reshape(g.n, -1)
    z = fo.solve(g.n, g.src, g.dst, g.w, s, tol=tol).reshape(g.n, -1)
    q = [fo.quantities_from_z(g.n, g.src, g.dst, g.w, s[:, j], z[:, j]) for j in range(s.shape[1])]
    return z, q


def test_p5_forest_matrix(ctx):
    from paper_2101_08143_gb300 import fj
    g = synth.path_graph(5)
    with ctx.upload_edges(g) as dg:
        om, _, info = ctx.solve(dg, np.eye(5), opts=fj.default_opts(tol=1e-13))
    expect = fo.forest_matrix(5, g.src, g.dst, g.w)
    np.testing.assert_allclose(om, expect, atol=1e-12)
    assert abs(om[0, 1] * 55 - 13) < 1e-10


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_erdos_renyi_2k(ctx, prec):
    """n = 2,000 ER graph, average degree 10, unit weights, s ~ U[0,1]."""
    from paper_2101_08143_gb300 import fj
    spec = synth.WORKLOADS["er_n2k_d10"]
    g = synth.make_graph(spec)
    s = synth.make_opinions(spec, g.n)[:, 0]
    zo, qo = _oracle(g, s)
    with ctx.upload_edges(g) as dg:
        assert dg.stats() == {"n": 2000, "nnz": 20000, "weighted": False}
        z, q, info = ctx.solve(dg, s, opts=fj.default_opts(precision=prec, tol=1e-10 if prec != 2 else 1e-6))
    _check_quantities(q[0], qo[0], s, TOL[prec])
    ztol = 1e-8 if prec != 2 else 1e-4
    np.testing.assert_allclose(z, zo[:, 0], atol=ztol)
    if prec != 2:
        assert info["rel_residual"] <= 1e-10
    assert info["iterations"] > 0


def test_bench_workload_full_size(ctx):
    """The benchmark's own workload and launch configuration: Chung-Lu
    n = 1,000,000, m = 5,000,000, exponent 2.3, weights U(0,1], one
    s ~ U[0,1]; device-pointer upload with FJ_MERGE_DUPLICATES, mixed
    precision to relative residual 1e-8 on the full grid.  Every z_i is
    compared with the oracle's float64 solve.  Since I + L has no eigenvalue
    below 1, ||z - z*|| <= ||s_bar - (I + L) q|| <= 1e-8 ||s_bar||, which bounds
    each element; the five quantities match to 1e-6."""
    import torch
    from paper_2101_08143_gb300 import fj
    spec = synth.WORKLOADS["cl_n1m_m5m_b2.3"]
    g = synth.make_graph(spec)
    s = synth.make_opinions(spec, g.n)[:, 0]
    zo, qo = _oracle(g, s)
    dev = torch.device("cuda")
    with ctx.upload(g.n, torch.from_numpy(g.src).to(dev), torch.from_numpy(g.dst).to(dev),
                    torch.from_numpy(g.w).to(dev), merge_duplicates=True) as dg:
        assert dg.stats()["nnz"] == 2 * g.m
        z, q, info = ctx.solve(dg, torch.from_numpy(s).to(dev),
                               opts=fj.default_opts(tol=1e-8, precision=fj.PREC_MIXED))
    assert info["rel_residual"] <= 1e-8
    bound = 1e-8 * float(np.linalg.norm(s - s.mean()))
    assert float(np.max(np.abs(z.cpu().numpy() - zo[:, 0]))) <= bound
    _check_quantities(q[0], qo[0], s, 1e-6)


def test_bench_workload_pure_float32(ctx):
    """The 1M-node bench graph in the pure float32 mode (one float32 PCG solve
    to relative residual 1e-6, no refinement): every quantity within 1e-3 of
    the oracle (the float32 tolerance)."""
    import torch
    from paper_2101_08143_gb300 import fj
    spec = synth.WORKLOADS["cl_n1m_m5m_b2.3"]
    g = synth.make_graph(spec)
    s = synth.make_opinions(spec, g.n)[:, 0]
    zo, qo = _oracle(g, s)
    dev = torch.device("cuda")
    with ctx.upload(g.n, torch.from_numpy(g.src).to(dev), torch.from_numpy(g.dst).to(dev),
                    torch.from_numpy(g.w).to(dev), merge_duplicates=True) as dg:
        z, q, info = ctx.solve(dg, torch.from_numpy(s).to(dev),
                               opts=fj.default_opts(tol=1e-6, precision=fj.PREC_FP32))
    assert info["refinements"] <= 1
    _check_quantities(q[0], qo[0], s, 1e-3)
    # ||z - z*|| <= ||s_bar - (I + L) q|| (no eigenvalue of I + L below 1)
    bound = 1.01 * info["rel_residual"] * float(np.linalg.norm(s - s.mean()))
    assert float(np.max(np.abs(z.cpu().numpy() - zo[:, 0]))) <= bound


@pytest.mark.parametrize("n,m,weighted,seed", [(300, 900, True, 1), (1000, 20000, True, 2),
                                               (4097, 9000, False, 3), (12345, 60000, True, 4)])
def test_random_graphs_several_tiles(ctx, n, m, weighted, seed):
    g = synth.erdos_renyi(n, m, seed=seed, weighted=weighted)
    s = synth.opinions_uniform(n, 1, seed)[:, 0]
    zo, qo = _oracle(g, s)
    with ctx.upload_edges(g) as dg:
        z, q, _ = ctx.solve(dg, s)
    _check_quantities(q[0], qo[0], s, 1e-6)
    np.testing.assert_allclose(z, zo[:, 0], atol=1e-8)


@pytest.mark.parametrize("k", [2, 3, 7, 33])
def test_multi_rhs(ctx, k):
    """k opinion vectors in one call (launches of 32/16/8/4/2/1 columns)."""
    g = synth.chung_lu(5000, 20000, 2.3, seed=11, weighted=True)
    s = synth.opinions_batch_mix(g.n, k, 5)
    zo, qo = _oracle(g, s)
    with ctx.upload_edges(g) as dg:
        z, q, _ = ctx.solve(dg, s)
    for j in range(k):
        _check_quantities(q[j], qo[j], s[:, j], 1e-6)
    np.testing.assert_allclose(z, zo, atol=1e-8)


def test_chung_lu_hubs(ctx):
    """Power-law graph whose hub rows span many tiles and warps."""
    g = synth.chung_lu(60_000, 300_000, 2.1, seed=7, weighted=True)
    s = synth.opinions_polarized(g.n, 1, 3)[:, 0]
    zo, qo = _oracle(g, s)
    with ctx.upload_edges(g) as dg:
        z, q, info = ctx.solve(dg, s)
    _check_quantities(q[0], qo[0], s, 1e-6)
    np.testing.assert_allclose(z, zo[:, 0], atol=1e-8)


@pytest.mark.parametrize("blocks", [1, 2, 5])
def test_launch_shapes_agree(ctx, blocks):
    """Small persistent grids (down to one block) give the same results."""
    g = synth.chung_lu(20_000, 80_000, 2.3, seed=8, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 4)[:, 0]
    zo, qo = _oracle(g, s)
    ctx.set_max_blocks(blocks)
    try:
        with ctx.upload_edges(g) as dg:
            z, q, _ = ctx.solve(dg, s)
    finally:
        ctx.set_max_blocks(0)
    _check_quantities(q[0], qo[0], s, 1e-6)
    np.testing.assert_allclose(z, zo[:, 0], atol=1e-8)


@pytest.mark.parametrize("blocks", [1, 3])
def test_launch_shapes_agree_wide(ctx, blocks):
    """A 16-column launch on grids of one and three blocks matches the oracle."""
    g = synth.chung_lu(20_000, 80_000, 2.3, seed=8, weighted=True)
    s = synth.opinions_uniform(g.n, 16, 4)
    zo, qo = _oracle(g, s)
    ctx.set_max_blocks(blocks)
    try:
        with ctx.upload_edges(g) as dg:
            z, q, _ = ctx.solve(dg, s)
    finally:
        ctx.set_max_blocks(0)
    for j in range(16):
        _check_quantities(q[j], qo[j], s[:, j], 1e-6)
    np.testing.assert_allclose(z, zo, atol=1e-8)


@pytest.mark.parametrize("grid", [1, 7, "2*SMs"])
@pytest.mark.parametrize("k", [1, 16])
def test_exact_grids(ctx, grid, k):
    """fj_set_grid runs the solve on exactly the given grid, including many
    more blocks than the work sizing picks (22 here), where most warps get no
    work unit; results match the oracle."""
    import torch
    g = synth.chung_lu(20_000, 80_000, 2.3, seed=8, weighted=True)
    s = synth.opinions_uniform(g.n, k, 4)
    zo, qo = _oracle(g, s)
    if grid == "2*SMs":
        grid = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    ctx.set_grid(grid)
    try:
        with ctx.upload_edges(g) as dg:
            z, q, info = ctx.solve(dg, s)
    finally:
        ctx.set_grid(0)
    assert info["blocks"] == grid
    for j in range(k):
        _check_quantities(q[j], qo[j], s[:, j], 1e-6)
    np.testing.assert_allclose(z, zo, atol=1e-8)


@pytest.mark.parametrize("k,prec", [(1, 1), (4, 0), (16, 0)])
def test_grid_tuner(ctx, k, prec):
    """fj_tune times the default sizing and grids of 2*SMs, SMs, ..., 1
    blocks, keeps the fastest, and later solves of as many columns in the
    same precision class run on it (the same bits as a solve on that grid
    set by hand); other column counts keep the default sizing; results match
    the oracle."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(20_000, 80_000, 2.3, seed=8, weighted=True)
    s = synth.opinions_uniform(g.n, k, 4)
    s_other = synth.opinions_uniform(g.n, k + 1, 5)
    zo, qo = _oracle(g, s)
    opts = fj.default_opts(precision=prec)
    with ctx.upload_edges(g) as dg:
        _, _, info0 = ctx.solve(dg, s, opts=opts)
        _, _, info_other0 = ctx.solve(dg, s_other, opts=opts)
        res = ctx.tune(dg, s, opts=opts, repeats=2)
        grids = [b for b, _ in res["grids"]]
        times = dict(res["grids"])
        assert grids[0] == 0 and grids[-1] == 1 and grids[1:] == sorted(grids[1:], reverse=True)
        assert all(ms > 0 for ms in times.values())
        assert times[res["best"]] == min(times.values())
        z_t, q_t, info_t = ctx.solve(dg, s, opts=opts)
        assert info_t["blocks"] == (res["best"] or info0["blocks"])
        _, _, info_other = ctx.solve(dg, s_other, opts=opts)
        assert info_other["blocks"] == info_other0["blocks"]
        ctx.set_grid(info_t["blocks"])
        try:
            z_e, q_e, _ = ctx.solve(dg, s, opts=opts)
        finally:
            ctx.set_grid(0)
        with pytest.raises(fj.FJError):
            ctx.tune(dg, s, opts=fj.default_opts(flags=fj.FJ_TWO_SOLVES))
    assert np.array_equal(z_t, z_e) and q_t == q_e
    for j in range(k):
        _check_quantities(q_t[j], qo[j], s[:, j], 1e-6)
    np.testing.assert_allclose(z_t, zo, atol=1e-8)


@pytest.mark.parametrize("k", [2, 40])
def test_deterministic_bits(ctx, k):
    """Repeated solves, and solves on a re-uploaded graph, give the same bits;
    k = 40 runs the 32- and 8-column launches, whose warps take work units
    in whatever order they become free."""
    g = synth.chung_lu(30_000, 120_000, 2.2, seed=9, weighted=True)
    s = synth.opinions_uniform(g.n, k, 6)
    with ctx.upload_edges(g) as dg:
        z1, q1, _ = ctx.solve(dg, s)
        z2, q2, _ = ctx.solve(dg, s)
    with ctx.upload_edges(g) as dg2:
        z3, q3, _ = ctx.solve(dg2, s)
    assert np.array_equal(z1, z2) and np.array_equal(z1, z3)
    assert q1 == q2 == q3


@pytest.mark.parametrize("k,prec", [(1, 0), (3, 0), (17, 0), (2, 1)])
def test_two_solves_mode_matches_algorithm_1(ctx, k, prec):
    """FJ_TWO_SOLVES runs Algorithm 1 as printed (z~ from s, q from s_bar;
    C_I = ||L z~||^2, D = ||W^1/2 B q||^2, P = ||q||^2, C = ||z~||^2) and
    matches the oracle's step-by-step Algorithm 1 and the definitions."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(8000, 40_000, 2.3, seed=21, weighted=True)
    s = synth.opinions_batch_mix(g.n, k, 7)
    zo, qo = _oracle(g, s)
    o = fj.default_opts(tol=1e-10, precision=prec, flags=fj.FJ_TWO_SOLVES)
    with ctx.upload_edges(g) as dg:
        z, q, info = ctx.solve(dg, s, opts=o)
        _, q1, _ = ctx.solve(dg, s, opts=fj.default_opts(tol=1e-10, precision=prec))
    assert info["rel_residual"] <= 1e-10
    for j in range(k):
        lit = fo.approxim(g.n, g.src, g.dst, g.w, s[:, j])
        _check_quantities(q[j], lit, s[:, j], 1e-6)
        _check_quantities(q[j], qo[j], s[:, j], 1e-6)
        _check_quantities(q[j], q1[j], s[:, j], 1e-6)
        assert q[j]["I_dc"] == pytest.approx(q[j]["D"] + q[j]["C"], rel=1e-15)
    np.testing.assert_allclose(z, zo, atol=1e-8)


@pytest.mark.parametrize("dist", ["uniform", "exponential", "power_law"])
@pytest.mark.parametrize("two", [False, True])
def test_paper_opinion_distributions(ctx, dist, two):
    """The paper's three opinion distributions (uniform, exponential and
    power law with exponent 2.5, each scaled to max 1, Sec. 5) on a power-law
    graph, in the default and the two-solve mode."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(12_000, 60_000, 2.2, seed=31, weighted=True)
    gen = {"uniform": synth.opinions_uniform, "exponential": synth.opinions_exponential,
           "power_law": synth.opinions_power_law}[dist]
    s = gen(g.n, 2, 13)
    zo, qo = _oracle(g, s)
    o = fj.default_opts(tol=1e-10, flags=fj.FJ_TWO_SOLVES if two else 0)
    with ctx.upload_edges(g) as dg:
        z, q, _ = ctx.solve(dg, s, opts=o)
    for j in range(2):
        _check_quantities(q[j], qo[j], s[:, j], 1e-6)
    np.testing.assert_allclose(z, zo, atol=1e-8)


@pytest.mark.parametrize("k,two", [(1, False), (5, False), (2, True)])
def test_warm_start(ctx, k, two):
    """fj_solve_warm: from the exact answer it stops at once; from the answer
    for a slightly changed s it needs fewer iterations than a cold solve and
    matches the oracle; from a poor guess it still converges."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(20_000, 100_000, 2.2, seed=41, weighted=True)
    s = synth.opinions_uniform(g.n, k, 8)
    o = fj.default_opts(tol=1e-10, flags=fj.FJ_TWO_SOLVES if two else 0)
    s2 = s.copy()
    rng = np.random.default_rng(2)
    idx = rng.choice(g.n, g.n // 100, replace=False)
    s2[idx] = rng.random((len(idx), k))  # 1% of the opinions change
    zo, qo = _oracle(g, s2)
    with ctx.upload_edges(g) as dg:
        z1, _, info1 = ctx.solve(dg, s, opts=o)
        _, _, again = ctx.solve(dg, s, opts=o, z0=z1)
        assert again["iterations"] == 0 and again["rel_residual"] <= 1e-10
        zc, qc, cold = ctx.solve(dg, s2, opts=o)
        zw, qw, warm = ctx.solve(dg, s2, opts=o, z0=z1)
        _, qp, poor = ctx.solve(dg, s2, opts=o, z0=-5.0 * np.ones_like(s2))
    assert warm["rel_residual"] <= 1e-10 and poor["rel_residual"] <= 1e-10
    assert warm["iterations"] < cold["iterations"]
    for j in range(k):
        for qq in (qw, qp, qc):
            _check_quantities(qq[j], qo[j], s2[:, j], 1e-6)
    np.testing.assert_allclose(zw, zo, atol=1e-8)


@pytest.mark.parametrize("weighted,merge", [(True, False), (False, False), (True, True)])
def test_largest_connected_component(ctx, weighted, merge):
    """fj_graph_lcc: the component's nodes (in increasing input id) match the
    oracle's, and solving on it matches the oracle on the induced subgraph;
    a graph of several components, isolated nodes and a hub row of several
    chunks.  With merge, a repeated pair survives as a parallel edge."""
    a = synth.chung_lu(9000, 40_000, 2.1, seed=51, weighted=weighted)
    b = synth.erdos_renyi(3000, 9000, seed=52, weighted=weighted)
    n = a.n + b.n + 500  # 500 isolated nodes
    rng = np.random.default_rng(5)
    relabel = rng.permutation(n)
    src = relabel[np.concatenate([a.src, b.src + a.n])].astype(np.int32)
    dst = relabel[np.concatenate([a.dst, b.dst + a.n])].astype(np.int32)
    w = np.concatenate([a.w, b.w]) if weighted else None
    if merge:
        src, dst = np.append(src, dst[0]), np.append(dst, src[0])
        w = np.append(w, np.float32(0.25)) if weighted else None
    nodes, s2, d2, w2 = fo.largest_component(n, src, dst, w)
    assert len(nodes) < a.n + 1
    s = synth.opinions_uniform(n, 2, 9)
    sl = s[nodes]
    zo, qo = _oracle_edges(len(nodes), s2, d2, w2, sl)
    with ctx.upload(n, src, dst, w, merge_duplicates=merge) as dg:
        with dg.lcc() as lg:
            st = lg.stats()
            assert st["n"] == len(nodes) and st["nnz"] == 2 * len(s2) and st["weighted"] == weighted
            np.testing.assert_array_equal(lg.node_ids(), nodes)
            z, q, _ = ctx.solve(lg, sl)
        np.testing.assert_array_equal(dg.node_ids(), np.arange(n))
    for j in range(2):
        _check_quantities(q[j], qo[j], sl[:, j], 1e-6)
    np.testing.assert_allclose(z, zo, atol=1e-8)


def test_lcc_of_an_edgeless_graph_is_node_zero(ctx):
    g = synth.edgeless(50)
    with ctx.upload_edges(g) as dg:
        with dg.lcc() as lg:
            assert lg.stats()["n"] == 1 and lg.stats()["nnz"] == 0
            assert list(lg.node_ids()) == [0]


def test_page_locked_host_edges(ctx):
    """Page-locked host edge arrays are read by the validation pass directly
    (mapped), pageable ones copied first: both give the same bits as a
    device-pointer upload, and bad edges are still rejected."""
    import torch
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(30_000, 150_000, 2.2, seed=61, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 4)[:, 0]
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    dev = torch.device("cuda")
    with ctx.upload(g.n, torch.from_numpy(g.src).to(dev), torch.from_numpy(g.dst).to(dev),
                    torch.from_numpy(g.w).to(dev)) as dg:
        z0, q0, _ = ctx.solve(dg, s)
    for src, dst, w in ((pin(g.src), pin(g.dst), pin(g.w)), (pin(g.src), g.dst, pin(g.w)),
                        (pin(g.src), pin(g.dst), None)):
        with ctx.upload(g.n, src, dst, w) as dg:
            z, q, _ = ctx.solve(dg, s)
        if w is not None:
            assert np.array_equal(z, z0) and q == q0
        else:
            zo, qo = _oracle_edges(g.n, g.src, g.dst, None, s)
            _check_quantities(q[0], qo[0], s, 1e-6)
    bad = pin(g.dst.copy())
    bad[1234] = g.n + 7
    with pytest.raises(fj.FJError) as e:
        ctx.upload(g.n, pin(g.src), bad, pin(g.w))
    assert e.value.code == fj.FJ_ERR_GRAPH and "edge 1234" in str(e.value)
    badw = pin(g.w.copy())
    badw[99] = -1.0
    with pytest.raises(fj.FJError) as e:
        ctx.upload(g.n, pin(g.src), pin(g.dst), badw)
    assert e.value.code == fj.FJ_ERR_GRAPH and "edge 99" in str(e.value)


def test_lcc_tie_goes_to_the_smallest_id(ctx):
    src = np.array([1, 2, 3, 4, 5, 0], np.int32)
    dst = np.array([2, 3, 1, 5, 0, 4], np.int32)
    with ctx.upload(7, src, dst) as dg:
        with dg.lcc() as lg:
            assert list(lg.node_ids()) == [0, 4, 5]
            assert lg.stats()["nnz"] == 6


def test_two_solves_and_warm_start_with_device_pointers(ctx):
    """Both modes through device-resident s, z and z0."""
    import torch
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(10_000, 50_000, 2.2, seed=71, weighted=True)
    s = synth.opinions_uniform(g.n, 3, 5)
    zo, qo = _oracle(g, s)
    dev = torch.device("cuda")
    sd = torch.from_numpy(np.ascontiguousarray(s.T)).to(dev)
    with ctx.upload_edges(g) as dg:
        z2, q2, _ = ctx.solve(dg, sd, opts=fj.default_opts(tol=1e-10, flags=fj.FJ_TWO_SOLVES))
        zw, qw, info = ctx.solve(dg, sd, opts=fj.default_opts(tol=1e-10), z0=z2)
    assert info["iterations"] == 0
    for j in range(3):
        _check_quantities(q2[j], qo[j], s[:, j], 1e-6)
        _check_quantities(qw[j], qo[j], s[:, j], 1e-6)
    np.testing.assert_allclose(z2.cpu().numpy().T, zo, atol=1e-8)
    np.testing.assert_allclose(zw.cpu().numpy().T, zo, atol=1e-8)


def test_two_solves_mode_rejected_where_unsupported(ctx):
    from paper_2101_08143_gb300 import fj
    g = synth.erdos_renyi(500, 2000, seed=4)
    o = fj.default_opts(flags=fj.FJ_TWO_SOLVES)
    with pytest.raises(fj.FJError) as e:
        fj.submit_edges(ctx, g.n, g.src, g.dst, None, np.ones(g.n), opts=o)
    assert e.value.code == fj.FJ_ERR_ARG


# ------------------------------------------------------------ edge cases

def test_opinions_outside_the_unit_interval_warn(ctx):
    """Any finite s is solved.  Opinions outside [0, 1], the range Sec. 2.2
    assumes, set FJ_WARN_OPINION_RANGE in the info of the direct and the
    served solve; in-range opinions leave it clear; results match the
    oracle either way."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(5_000, 20_000, 2.3, seed=3, weighted=True)
    s_in = synth.opinions_uniform(g.n, 2, 7)
    s_out = s_in.copy()
    s_out[:, 1] = 3.0 * s_in[:, 1] - 1.0  # second column in [-1, 2]
    zo, qo = _oracle(g, s_out)
    with ctx.upload_edges(g) as dg:
        _, _, info_in = ctx.solve(dg, s_in)
        z, q, info_out = ctx.solve(dg, s_out)
        t = fj.submit(ctx, dg, s_out)
        rc, q_srv, info_srv = fj.poll(ctx, t, timeout_us=30_000_000)
    assert info_in["warnings"] == 0
    assert info_out["warnings"] == fj.FJ_WARN_OPINION_RANGE
    assert rc == fj.FJ_OK and info_srv["warnings"] == fj.FJ_WARN_OPINION_RANGE
    for j in range(2):
        _check_quantities(q[j], qo[j], s_out[:, j], 1e-6)
        _check_quantities(q_srv[j], qo[j], s_out[:, j], 1e-6)
    np.testing.assert_allclose(z, zo, atol=1e-8)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_opinions_are_a_numeric_error(ctx, bad):
    """A NaN or infinite s_i makes the float64 residual non-finite at the
    first check: every block sees the same reduced value, stops, and the call
    returns FJ_ERR_NUMERIC."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(5_000, 20_000, 2.3, seed=3, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 7)[:, 0].copy()
    s[123] = bad
    with ctx.upload_edges(g) as dg:
        with pytest.raises(fj.FJError) as e:
            ctx.solve(dg, s)
        assert e.value.code == fj.FJ_ERR_NUMERIC
        # the context stays usable
        s[123] = 0.5
        _, q, info = ctx.solve(dg, s)
    assert info["rc"] == fj.FJ_OK


def test_edgeless_graph(ctx):
    g = synth.edgeless(1000)
    s = synth.opinions_uniform(1000, 1, 1)[:, 0]
    with ctx.upload_edges(g) as dg:
        z, q, _ = ctx.solve(dg, s)
    np.testing.assert_allclose(z, s, atol=1e-14)
    assert q[0]["C_I"] < 1e-20 and q[0]["D"] == 0.0
    assert q[0]["C"] == pytest.approx(float(np.sum(s ** 2)), rel=1e-13)


def test_single_node(ctx):
    with ctx.upload(1, np.zeros(0, np.int32), np.zeros(0, np.int32)) as dg:
        z, q, _ = ctx.solve(dg, np.array([0.7]))
    assert z[0] == pytest.approx(0.7)
    assert q[0]["P"] == 0.0 and q[0]["C"] == pytest.approx(0.49)


def test_constant_opinions(ctx):
    g = synth.erdos_renyi(3000, 12000, seed=2, weighted=True)
    s = np.full(3000, 0.25)
    with ctx.upload_edges(g) as dg:
        z, q, info = ctx.solve(dg, s)
    np.testing.assert_allclose(z, 0.25, atol=1e-15)
    assert q[0]["P"] < 1e-25 and q[0]["D"] < 1e-25 and q[0]["C_I"] < 1e-25


def test_self_loops_and_parallel_edges(ctx):
    """Self-loops vanish; with FJ_MERGE_DUPLICATES repeated pairs add their
    weights, without it they are rejected."""
    from paper_2101_08143_gb300 import fj
    src = np.array([0, 1, 0, 2, 2, 3, 3], np.int32)
    dst = np.array([1, 2, 1, 2, 3, 3, 0], np.int32)
    w = np.array([0.5, 1.0, 0.25, 9.0, 2.0, 4.0, 0.125], np.float32)
    s = np.array([0.9, 0.1, 0.4, 0.7])
    expect = fo.solve_dense(4, src, dst, w, s)
    with ctx.upload(4, src, dst, w, merge_duplicates=True) as dg:
        assert dg.stats()["nnz"] == 10
        z, _, _ = ctx.solve(dg, s)
    np.testing.assert_allclose(z, expect, atol=1e-12)
    with pytest.raises(fj.FJError) as e:
        ctx.upload(4, src, dst, w)
    assert e.value.code == fj.FJ_ERR_GRAPH and "(0, 1)" in str(e.value)
    # self-loops alone are not repeats
    with ctx.upload(4, src[[1, 3, 4, 5, 6]], dst[[1, 3, 4, 5, 6]], w[[1, 3, 4, 5, 6]]) as dg:
        assert dg.stats()["nnz"] == 6


@pytest.mark.parametrize("hub", [False, True])
def test_repeated_pair_found_in_short_and_long_rows(ctx, hub):
    """A pair listed a second time, reversed, is reported with its input ids,
    both when its rows are short (sliced ELL) and when one of them is a hub
    row of several chunks."""
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(20_000, 100_000, 2.1, seed=12, weighted=True)
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    if hub:
        u = int(np.argmax(deg))
        e = int(np.nonzero((g.src == u) | (g.dst == u))[0][len(g.src) // 7 % int(deg[u])])
        assert deg[u] > 1024
    else:
        e = int(np.nonzero((deg[g.src] <= 64) & (deg[g.dst] <= 64))[0][0])
    a, b = int(g.src[e]), int(g.dst[e])
    src = np.append(g.src, b).astype(np.int32)
    dst = np.append(g.dst, a).astype(np.int32)
    w = np.append(g.w, np.float32(0.5))
    with pytest.raises(fj.FJError) as err:
        ctx.upload(g.n, src, dst, w)
    assert err.value.code == fj.FJ_ERR_GRAPH
    assert f"({min(a, b)}, {max(a, b)})" in str(err.value)
    # merged: the pair's weight is the sum
    s = synth.opinions_uniform(g.n, 1, 3)[:, 0]
    zo = fo.solve(g.n, src, dst, w, s)
    with ctx.upload(g.n, src, dst, w, merge_duplicates=True) as dg:
        z, _, _ = ctx.solve(dg, s)
    np.testing.assert_allclose(z, zo, atol=1e-8)


def test_disconnected_components(ctx):
    a = synth.erdos_renyi(500, 2000, seed=3, weighted=True)
    src = np.concatenate([a.src, a.src + 500])
    dst = np.concatenate([a.dst, a.dst + 500])
    w = np.concatenate([a.w, a.w * 0.5])
    s = synth.opinions_uniform(1000, 1, 2)[:, 0]
    zo = fo.solve(1000, src, dst, w, s)
    with ctx.upload(1000, src, dst, w) as dg:
        z, _, _ = ctx.solve(dg, s)
    np.testing.assert_allclose(z, zo, atol=1e-9)
    assert z[:500].sum() == pytest.approx(s[:500].sum(), rel=1e-10)


def test_bad_graphs_rejected(ctx):
    from paper_2101_08143_gb300 import fj
    with pytest.raises(fj.FJError) as e:
        ctx.upload(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32))
    assert e.value.code == fj.FJ_ERR_GRAPH
    with pytest.raises(fj.FJError) as e:
        ctx.upload(3, np.array([0], np.int32), np.array([1], np.int32), np.array([0.0], np.float32))
    assert e.value.code == fj.FJ_ERR_GRAPH
    with pytest.raises(fj.FJError) as e:
        ctx.upload(3, np.array([0], np.int32), np.array([1], np.int32), np.array([np.nan], np.float32))
    assert e.value.code == fj.FJ_ERR_GRAPH
    with pytest.raises(fj.FJError) as e:
        ctx.upload(0, np.array([], np.int32), np.array([], np.int32))
    assert e.value.code == fj.FJ_ERR_ARG


def test_not_converged_reported(ctx):
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(20_000, 80_000, 2.3, seed=8, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 4)[:, 0]
    with ctx.upload_edges(g) as dg:
        _, q, info = ctx.solve(dg, s, opts=fj.default_opts(max_iter=3), raise_on_error=False)
    assert info["rc"] == fj.FJ_ERR_NOT_CONVERGED
    assert info["iterations"] <= 3


def test_device_pointers(ctx):
    """s and z as torch CUDA tensors (column-major: shape (k, n))."""
    import torch
    g = synth.erdos_renyi(5000, 25000, seed=5, weighted=True)
    s = synth.opinions_uniform(g.n, 3, 9)
    zo, qo = _oracle(g, s)
    sd = torch.from_numpy(np.ascontiguousarray(s.T)).cuda()
    with ctx.upload(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                    torch.from_numpy(g.w).cuda()) as dg:
        z, q, _ = ctx.solve(dg, sd)
    np.testing.assert_allclose(z.cpu().numpy().T, zo, atol=1e-8)
    for j in range(3):
        _check_quantities(q[j], qo[j], s[:, j], 1e-6)


def test_host_z_out_one_and_two_dimensional(ctx):
    """A caller's host z_out, 1-D for one opinion vector or n x k Fortran
    order, receives z in place."""
    g = synth.erdos_renyi(2000, 8000, seed=141, weighted=True)
    s = synth.opinions_uniform(g.n, 2, 142)
    zo, _ = _oracle(g, s)
    with ctx.upload_edges(g) as dg:
        z1 = np.empty(g.n)
        z, _, _ = ctx.solve(dg, np.ascontiguousarray(s[:, 0]), z_out=z1)
        assert z is z1
        np.testing.assert_allclose(z1, zo[:, 0], atol=1e-8)
        z2 = np.empty((g.n, 2), order="F")
        z, _, _ = ctx.solve(dg, s, z_out=z2)
        assert z is z2
        np.testing.assert_allclose(z2, zo, atol=1e-8)
