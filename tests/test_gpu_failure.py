"""The bounded grid barrier: a solve whose barrier wait runs out returns
FJ_ERR_TIMEOUT, and the context (and the serving worker) stays usable.

The failure is made without faulting or hanging the GPU: the library's test
hook fj_debug_barrier shortens every barrier wait to 20 ms and makes block 0
of the next multi-block solve skip its arrival at one barrier, so the other
blocks wait on a count that never completes until their limit runs out.
"""
import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth

pytestmark = pytest.mark.gpu

WAIT_NS = 20_000_000  # 20 ms


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08143_gb300 import fj
    lib = fj.load()
    c = fj.Context(0)
    yield fj, lib, c
    lib.fj_debug_barrier(0, 0)
    c.close()


def _graph_and_oracle():
    g = synth.chung_lu(20000, 100000, 2.3, seed=21, weighted=True)
    s = synth.opinions_uniform(g.n, 1, 22)[:, 0]
    z = fo.solve(g.n, g.src, g.dst, g.w, s)
    return g, s, fo.quantities_from_z(g.n, g.src, g.dst, g.w, s, z)


def _check(q, qo, s):
    for name in fo.QUANTITY_NAMES:
        assert fo.relative_error(qo[name], q[name], 1e-12 * float(s @ s)) <= 1e-6, name


@pytest.mark.parametrize("withhold", [1, 3, 6])
def test_barrier_timeout_then_a_normal_solve(env, withhold):
    fj, lib, ctx = env
    g, s, qo = _graph_and_oracle()
    with ctx.upload_edges(g) as dg:
        ctx.set_grid(8)
        try:
            assert lib.fj_debug_barrier(WAIT_NS, withhold) == fj.FJ_OK
            _, _, info = ctx.solve(dg, s, raise_on_error=False)
            assert info["rc"] == fj.FJ_ERR_TIMEOUT, info
            assert b"timed out" in lib.fj_last_error()
            assert info["blocks"] == 8
        finally:
            lib.fj_debug_barrier(0, 0)
            ctx.set_grid(0)
        _, q, info = ctx.solve(dg, s)
    assert info["rc"] == fj.FJ_OK
    _check(q[0], qo, s)


def test_served_request_times_out_and_the_next_one_completes(env):
    fj, lib, ctx = env
    g, s, qo = _graph_and_oracle()
    fj.serve_config(ctx, max_inflight=4, max_blocks_per_request=8)
    with ctx.upload_edges(g) as dg:
        try:
            assert lib.fj_debug_barrier(WAIT_NS, 2) == fj.FJ_OK
            t = fj.submit(ctx, dg, s)
            rc, _, _ = fj.poll(ctx, t, -1)
            assert rc == fj.FJ_ERR_TIMEOUT
        finally:
            lib.fj_debug_barrier(0, 0)
        t = fj.submit(ctx, dg, s)
        rc, q, _ = fj.poll(ctx, t, -1)
        assert rc == fj.FJ_OK
    _check(q[0], qo, s)
    fj.serve_config(ctx, max_inflight=16, max_blocks_per_request=0)


def test_hook_arguments_are_checked(env):
    fj, lib, _ = env
    assert lib.fj_debug_barrier(10, 0) == fj.FJ_ERR_ARG
    assert lib.fj_debug_barrier(0, -1) == fj.FJ_ERR_ARG
    assert lib.fj_debug_barrier(0, 0) == fj.FJ_OK
