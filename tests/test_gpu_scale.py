"""Parity at opinion scales far from the unit interval.

The mixed-precision refinement runs in double-float, whose exponent range is
float32's.  The solver therefore scales each right-hand side by an exact power
of two before the solve (the system (I + L) q = s_bar is linear, Eq. FJmodel02)
and scales z and the quantities back.  These tests run opinions multiplied by
2^-90, 2^-50 and 2^70 (exact in float64), and one call whose columns have
different scales, in every precision mode, against the float64 oracle run on
the same scaled opinions.  The quantities scale with the square of the factor
(Sec. 3.2 definitions), which the last test checks on the GPU alone.
"""
import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-6, 1: 1e-6, 2: 1e-3}  # relative error per quantity, by precision mode
SCALES = [2.0 ** -90, 2.0 ** -50, 2.0 ** 70]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08143_gb300 import fj
    c = fj.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def graph():
    return synth.chung_lu(5000, 20000, 2.3, seed=11, weighted=True)


def _oracle(g, s):
    s = s.reshape(g.n, -1)
    z = fo.solve(g.n, g.src, g.dst, g.w, s).reshape(g.n, -1)
    q = [fo.quantities_from_z(g.n, g.src, g.dst, g.w, s[:, j], z[:, j]) for j in range(s.shape[1])]
    return z, q


def _check(gq, oq, s, rtol):
    floor = 1e-12 * float(np.sum(s ** 2))
    for name in fo.QUANTITY_NAMES:
        err = fo.relative_error(oq[name], gq[name], floor=floor)
        assert err <= rtol, (name, gq[name], oq[name], err)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("scale", SCALES)
def test_scaled_opinions(ctx, graph, prec, scale):
    from paper_2101_08143_gb300 import fj
    g = graph
    s = synth.opinions_uniform(g.n, 1, 5)[:, 0] * scale
    zo, qo = _oracle(g, s)
    tol = 1e-10 if prec != 2 else 1e-6
    with ctx.upload_edges(g) as dg:
        z, q, info = ctx.solve(dg, s, opts=fj.default_opts(precision=prec, tol=tol))
    assert info["rel_residual"] <= tol
    assert info["iterations"] > 0
    _check(q[0], qo[0], s, TOL[prec])
    ztol = (1e-8 if prec != 2 else 1e-4) * scale
    np.testing.assert_allclose(z, zo[:, 0], rtol=0, atol=ztol)


@pytest.mark.parametrize("prec", [0, 1])
def test_columns_of_different_scales(ctx, graph, prec):
    """k = 4 in one launch: columns scaled by 2^-90, 1, 2^70 and 2^-50."""
    from paper_2101_08143_gb300 import fj
    g = graph
    f = np.array([2.0 ** -90, 1.0, 2.0 ** 70, 2.0 ** -50])
    s = np.asfortranarray(synth.opinions_uniform(g.n, 4, 6) * f[None, :])
    zo, qo = _oracle(g, s)
    with ctx.upload_edges(g) as dg:
        z, q, info = ctx.solve(dg, s, opts=fj.default_opts(precision=prec, tol=1e-10))
    assert info["rel_residual"] <= 1e-10
    for j in range(4):
        _check(q[j], qo[j], s[:, j], 1e-6)
        np.testing.assert_allclose(z[:, j], zo[:, j], rtol=0, atol=1e-8 * f[j])


def test_quantities_scale_with_the_square(ctx, graph):
    """Exact power-of-two scaling: the GPU's quantities at 2^70 s are 2^140
    times those at s, to the solve's tolerance (the iteration runs on the same
    scaled right-hand side, so they agree far more closely in practice)."""
    from paper_2101_08143_gb300 import fj
    g = graph
    s = synth.opinions_uniform(g.n, 1, 7)[:, 0]
    with ctx.upload_edges(g) as dg:
        o = fj.default_opts(tol=1e-10)
        z1, q1, _ = ctx.solve(dg, s, opts=o)
        z2, q2, _ = ctx.solve(dg, s * 2.0 ** 70, opts=o)
    for name in fo.QUANTITY_NAMES:
        assert q2[0][name] == pytest.approx(q1[0][name] * 2.0 ** 140, rel=1e-12), name
    np.testing.assert_allclose(z2, z1 * 2.0 ** 70, rtol=1e-12, atol=0)
