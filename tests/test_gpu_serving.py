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


def _overlapping_pairs(infos):
    iv = sorted((i["t_begin_ms"], i["t_end_ms"]) for i in infos)
    return sum(1 for a in range(len(iv)) for b in range(a + 1, len(iv))
               if iv[b][0] < iv[a][1] and iv[a][0] < iv[b][1])


@pytest.mark.parametrize("pack", [True, False])
def test_alone_and_in_a_mix_give_the_same_bits(ctx, pack):
    """The same request alone and amid 16 others gives the same bits, in
    packed batches or in its own launch; the requests' device intervals
    (admission to completion) overlap, i.e. their work shared the GPU."""
    from paper_2101_08143_gb300 import fj
    fj.serve_pack(ctx, 1 << 17 if pack else 0)
    try:
        g = synth.chung_lu(20_000, 100_000, 2.2, seed=77, weighted=True)
        s = synth.opinions_uniform(g.n, 3, 78)
        with ctx.upload_edges(g) as dg:
            rc, alone, info0 = fj.poll(ctx, fj.submit(ctx, dg, s), -1)
            assert rc == fj.FJ_OK
            assert info0["batched"] == (1 if pack else 0)
            others = _requests(2, 16)
            mix = [fj.submit_edges(ctx, h.n, h.src, h.dst, h.w, t) for h, t in others[:8]]
            mine = fj.submit(ctx, dg, s)
            mix += [fj.submit_edges(ctx, h.n, h.src, h.dst, h.w, t) for h, t in others[8:]]
            rc, in_mix, info1 = fj.poll(ctx, mine, -1)
            assert rc == fj.FJ_OK
            infos = [info1]
            for t in mix:
                rc, _, info = fj.poll(ctx, t, -1)
                assert rc == fj.FJ_OK
                infos.append(info)
        assert alone == in_mix
        assert info0["blocks"] == info1["blocks"]
        for i in infos:
            assert 0 < i["t_begin_ms"] < i["t_end_ms"]
        assert _overlapping_pairs(infos) >= 1
        _check(in_mix, g, s)
    finally:
        fj.serve_pack(ctx, 0)


def test_packed_and_own_launch_give_the_same_bits(ctx):
    """A small request solved in a packed batch and in its own launch: the
    same block count, the same bits (k = 13: parts of 8, 4 and 1 columns)."""
    from paper_2101_08143_gb300 import fj
    g = synth.erdos_renyi(5000, 30_000, seed=81, weighted=True)
    s = synth.opinions_uniform(g.n, 13, 82)
    out = []
    try:
        for pack in (1 << 17, 0):
            fj.serve_pack(ctx, pack)
            rc, q, info = fj.poll(ctx, fj.submit_edges(ctx, g.n, g.src, g.dst, g.w, s), -1)
            assert rc == fj.FJ_OK
            out.append((q, info))
    finally:
        fj.serve_pack(ctx, 0)
    assert out[0][1]["batched"] == 1 and out[1][1]["batched"] == 0
    assert out[0][1]["blocks"] == out[1][1]["blocks"]
    assert out[0][0] == out[1][0]
    _check(out[0][0], g, s)


def test_a_large_request_is_passed_over_at_most_32_times(ctx):
    """With the memory budget partly held, a large request that does not fit
    waits while later small ones are admitted ahead of it, but no more than
    32 of them; then nothing more is admitted until it fits, and it
    completes."""
    from paper_2101_08143_gb300 import fj
    # a request of n = 50,000 needs about 47 MB of the budget, the large one
    # about 185 MB: with any small request in flight the large one does not
    # fit a 200 MB budget.  The first small request runs 3000 inner
    # iterations (targets float32 and float64 cannot reach), so it holds its
    # memory while the others pass.
    small = [synth.erdos_renyi(50_000, 250_000, seed=300 + i, weighted=True) for i in range(4)]
    big = synth.chung_lu(200_000, 1_000_000, 2.3, seed=301, weighted=True)
    fj.serve_config(ctx, max_inflight=8, mem_budget_bytes=200_000_000)
    fj.serve_pack(ctx, 0)
    try:
        def sub(g, seed, opts=None):
            return fj.submit_edges(ctx, g.n, g.src, g.dst, g.w, synth.opinions_uniform(g.n, 1, seed)[:, 0],
                                   opts=opts)
        slow = sub(small[0], 0, fj.default_opts(tol=1e-300, inner_tol=1e-30, max_iter=3000, max_refine=1000))
        t_big = sub(big, 99)
        after = [sub(small[i % 4], 100 + i) for i in range(60)]
        rc, _, info_slow = fj.poll(ctx, slow, -1)
        assert rc == fj.FJ_ERR_NOT_CONVERGED
        infos = {}
        for t in [t_big] + after:
            rc, _, info = fj.poll(ctx, t, -1)
            assert rc == fj.FJ_OK
            infos[t.id] = info
        tb = infos[t_big.id]["t_begin_ms"]
        ahead = sum(1 for t in after if infos[t.id]["t_begin_ms"] < tb)
        assert 1 <= ahead <= 32, ahead
        # the large request did not start while the slow one held the memory
        assert tb >= info_slow["t_end_ms"]
    finally:
        fj.serve_config(ctx, max_inflight=16, mem_budget_bytes=8 << 30)
        fj.serve_pack(ctx, 0)


@pytest.mark.slow
def test_served_requests_of_a_million_nodes(ctx):
    """Requests of the serving workload's largest size (n up to 10^6), in a
    mix with small ones, against the oracle."""
    from paper_2101_08143_gb300 import fj
    bigs = [synth.chung_lu(300_000, 1_800_000, 2.2, seed=401, weighted=True),
            synth.erdos_renyi(1_000_000, 6_000_000, seed=402, weighted=True)]
    reqs = [(g, synth.opinions_uniform(g.n, 2, 410 + i)) for i, g in enumerate(bigs)]
    reqs += _requests(5, 6)
    tickets = [fj.submit_edges(ctx, g.n, g.src, g.dst, g.w, s, merge_duplicates=True) for g, s in reqs]
    for (g, s), t in zip(reqs, tickets):
        rc, q, info = fj.poll(ctx, t, -1)
        assert rc == fj.FJ_OK
        assert info["rel_residual"] <= 1e-10
        _check(q, g, s)


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
