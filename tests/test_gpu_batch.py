"""fj_solve_batch: many small graphs packed into shared persistent launches.

Each problem's parts run on their own block range of a packed launch, so a
part's results must be the same bits as the same part solved alone on as many
blocks (fj_set_grid), and every problem matches the float64 oracle at the
mixed-precision tolerance (1e-6 per quantity, Sec. 5's sigma).
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


def _problems(count, seed, ks=(1, 2, 3, 5, 8, 13, 16)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(10 ** rng.uniform(2.3, 4.3))
        m = max(1, int(n * rng.uniform(2, 10) / 2))
        if rng.random() < 0.5:
            g = synth.erdos_renyi(n, m, seed=seed * 100 + i, weighted=bool(rng.random() < 0.7))
        else:
            g = synth.chung_lu(n, m, rng.uniform(2.1, 2.5), seed=seed * 100 + i, weighted=True)
        k = int(ks[i % len(ks)])
        out.append((g, synth.opinions_uniform(g.n, k, seed * 100 + i)))
    return out


def _check(g, s, z, q, tol=1e-6, ztol=1e-8):
    zo = fo.solve(g.n, g.src, g.dst, g.w, s).reshape(g.n, -1)
    for j in range(s.shape[1]):
        qo = fo.quantities_from_z(g.n, g.src, g.dst, g.w, s[:, j], zo[:, j])
        for name in fo.QUANTITY_NAMES:
            err = fo.relative_error(qo[name], q[j][name], 1e-12 * float(s[:, j] @ s[:, j]))
            assert err <= tol, (name, j, q[j][name], qo[name])
    np.testing.assert_allclose(z, zo, rtol=0, atol=ztol)


def test_batch_matches_the_oracle(ctx):
    """40 problems of 7 widths: more parts than one launch packs."""
    probs = _problems(40, 1)
    graphs = [ctx.upload_edges(g) for g, _ in probs]
    try:
        rc, out = ctx.solve_batch(graphs, [s for _, s in probs])
        assert rc == 0
        for (g, s), (z, q, info) in zip(probs, out):
            assert info["status"] == 0 and info["rel_residual"] <= 1e-10
            assert info["blocks"] >= 1
            _check(g, s, z, q)
    finally:
        for dg in graphs:
            dg.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_parts_are_the_bits_of_a_solve_alone(ctx, prec):
    """Single-width problems (k in 1, 2, 4, 8, 16): each problem's results in
    the packed launch equal, bit for bit, fj_solve_ex on the same number of
    blocks."""
    from paper_2101_08143_gb300 import fj
    probs = _problems(20, 2, ks=(1, 2, 4, 8, 16))
    graphs = [ctx.upload_edges(g) for g, _ in probs]
    o = fj.default_opts(precision=prec)
    try:
        rc, out = ctx.solve_batch(graphs, [s for _, s in probs], opts=o)
        assert rc == 0
        for dg, (g, s), (z, q, info) in zip(graphs, probs, out):
            ctx.set_grid(info["blocks"])
            try:
                z1, q1, info1 = ctx.solve(dg, s, opts=o)
            finally:
                ctx.set_grid(0)
            assert info1["blocks"] == info["blocks"]
            assert np.array_equal(z1, z)
            assert q1 == q
            assert info1["iterations"] == info["iterations"]
    finally:
        for dg in graphs:
            dg.free()


def test_batch_with_device_pointers(ctx):
    import torch
    probs = _problems(12, 3)
    graphs = [ctx.upload_edges(g) for g, _ in probs]
    try:
        sd = [torch.from_numpy(np.ascontiguousarray(s.T)).cuda() for _, s in probs]
        rc, out = ctx.solve_batch(graphs, sd)
        assert rc == 0
        for (g, s), (z, q, _) in zip(probs, out):
            _check(g, s, z.cpu().numpy().T, q)
    finally:
        for dg in graphs:
            dg.free()


def test_one_bad_problem_does_not_spoil_the_others(ctx):
    """A NaN opinion makes its own problem FJ_ERR_NUMERIC; the other problems
    in the same packed launches still match the oracle."""
    from paper_2101_08143_gb300 import fj
    probs = _problems(6, 4, ks=(1, 2, 1, 4, 1, 2))
    s_bad = probs[2][1].copy()
    s_bad[5, 0] = np.nan
    graphs = [ctx.upload_edges(g) for g, _ in probs]
    try:
        s_list = [s for _, s in probs]
        s_list[2] = s_bad
        rc, out = ctx.solve_batch(graphs, s_list, raise_on_error=False)
        assert rc == fj.FJ_ERR_NUMERIC
        for i, ((g, s), (z, q, info)) in enumerate(zip(probs, out)):
            if i == 2:
                assert info["status"] == fj.FJ_ERR_NUMERIC
            else:
                assert info["status"] == 0
                _check(g, s, z, q)
    finally:
        for dg in graphs:
            dg.free()


def test_batch_arguments_are_checked(ctx):
    from paper_2101_08143_gb300 import fj
    lib = fj.load()
    assert lib.fj_solve_batch(ctx.handle, 0, None, None, None, None, None, None, None) == fj.FJ_ERR_ARG
    assert lib.fj_solve_batch(None, 1, None, None, None, None, None, None, None) == fj.FJ_ERR_ARG
