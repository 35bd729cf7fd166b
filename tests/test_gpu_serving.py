"""fj_submit / fj_poll: continuous batching of solve requests.

Each request's quantities are checked against the FP64 oracle, and a request
solved alone must give the same bits when it runs in a mix of others.
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


def _check(q, g, s, rtol=1e-6):
    s = np.asarray(s).reshape(g.n, -1)
    for j in range(s.shape[1]):
        z = fo.solve(g.n, g.src, g.dst, g.w, s[:, j])
        oq = fo.quantities_from_z(g.n, g.src, g.dst, g.w, s[:, j], z)
        floor = 1e-12 * float(np.sum(s[:, j] ** 2))
        for name in fo.QUANTITY_NAMES:
            assert fo.relative_error(oq[name], q[j][name], floor) <= rtol, (name, q[j][name], oq[name])


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(10 ** rng.uniform(3, 4.3))
        deg = rng.uniform(4, 20)
        m = int(n * deg / 2)
        if rng.random() < 0.5:
            g = synth.erdos_renyi(n, m, seed=1000 + i, weighted=True)
        else:
            g = synth.chung_lu(n, m, rng.uniform(2.1, 2.5), seed=1000 + i, weighted=True)
        k = int(rng.integers(1, 5))
        out.append((g, synth.opinions_uniform(n, k, 50 + i)))
    return out


def test_inline_requests_match_oracle(ctx):
    from paper_2101_08143_gb300 import fj
    reqs = _requests(1, 12)
    tickets = [fj.submit_edges(ctx, g.n, g.src, g.dst, g.w, s) for g, s in reqs]
    for (g, s), t in zip(reqs, tickets):
        rc, q, info = fj.poll(ctx, t, -1)
        assert rc == fj.FJ_OK
        assert info["rel_residual"] <= 1e-10
        _check(q, g, s)


def test_alone_and_in_a_mix_give_the_same_bits(ctx):
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(20_000, 100_000, 2.2, seed=77, weighted=True)
    s = synth.opinions_uniform(g.n, 3, 78)
    with ctx.upload_edges(g) as dg:
        rc, alone, _ = fj.poll(ctx, fj.submit(ctx, dg, s), -1)
        assert rc == fj.FJ_OK
        others = _requests(2, 16)
        mix = [fj.submit_edges(ctx, h.n, h.src, h.dst, h.w, t) for h, t in others[:8]]
        mine = fj.submit(ctx, dg, s)
        mix += [fj.submit_edges(ctx, h.n, h.src, h.dst, h.w, t) for h, t in others[8:]]
        rc, in_mix, _ = fj.poll(ctx, mine, -1)
        assert rc == fj.FJ_OK
        for t in mix:
            assert fj.poll(ctx, t, -1)[0] == fj.FJ_OK
    assert alone == in_mix
    _check(in_mix, g, s)


def test_serving_errors(ctx):
    from paper_2101_08143_gb300 import fj
    # a bad node id is found when the request's graph is built
    t = fj.submit_edges(ctx, 3, np.array([0, 5]), np.array([1, 1]), None, np.ones(3))
    rc, _, info = fj.poll(ctx, t, -1)
    assert rc == fj.FJ_ERR_GRAPH
    # a collected ticket is gone
    assert fj.poll(ctx, t, 0)[0] == fj.FJ_ERR_TICKET
    # a repeated pair fails the request unless merged
    src, dst = np.array([0, 1, 1]), np.array([1, 2, 0])
    t = fj.submit_edges(ctx, 3, src, dst, None, np.array([0.2, 0.5, 0.9]))
    assert fj.poll(ctx, t, -1)[0] == fj.FJ_ERR_GRAPH
    t = fj.submit_edges(ctx, 3, src, dst, None, np.array([0.2, 0.5, 0.9]), merge_duplicates=True)
    assert fj.poll(ctx, t, -1)[0] == fj.FJ_OK
    # a request larger than the whole budget is refused at submit
    fj.serve_config(ctx, mem_budget_bytes=1 << 20)
    g = synth.erdos_renyi(50_000, 200_000, seed=3)
    with pytest.raises(fj.FJError) as e:
        fj.submit_edges(ctx, g.n, g.src, g.dst, None, np.ones(g.n))
    assert e.value.code == fj.FJ_ERR_ADMIT
    fj.serve_config(ctx, mem_budget_bytes=8 << 30)


def test_pending_then_done(ctx):
    from paper_2101_08143_gb300 import fj
    g = synth.chung_lu(200_000, 1_000_000, 2.3, seed=5, weighted=True)
    s = synth.opinions_uniform(g.n, 2, 6)
    t = fj.submit_edges(ctx, g.n, g.src, g.dst, g.w, s)
    rc, _, _ = fj.poll(ctx, t, 0)
    assert rc in (fj.FJ_PENDING, fj.FJ_OK)
    if rc == fj.FJ_PENDING:
        rc, q, info = fj.poll(ctx, t, -1)
        assert rc == fj.FJ_OK
        assert info["device_ms"] > 0
