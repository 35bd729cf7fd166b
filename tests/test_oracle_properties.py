"""Property-based pins of the oracle on random small weighted graphs (CPU).

For every drawn graph and opinion vector:
  * the dense solve and the float64 CG solve agree (two independent routes to
    z = (I + L)^-1 s, Eq. FJmodel02);
  * the five quantities by their definitions (Sec. 3.2) equal the quadratic
    forms of Proposition 1 and the squared norms of Lemma PropA;
  * D + C = s^T z (Sec. 3.2) and C_I + 2D + C = ||s||^2 (from s - z = L z);
  * 1^T z = 1^T s (Sec. 3.1) and min s <= z_i <= max s (Omega is doubly
    stochastic and non-negative, Sec. 2.2).
Parallel edges, self-loops and isolated nodes are all allowed in the draw."""
import numpy as np
import pytest

import oracle.fj_oracle as fo

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


@st.composite
def graphs(draw):
    n = draw(st.integers(min_value=1, max_value=24))
    m = draw(st.integers(min_value=0, max_value=3 * n))
    src = np.array(draw(st.lists(st.integers(0, n - 1), min_size=m, max_size=m)), dtype=np.int32)
    dst = np.array(draw(st.lists(st.integers(0, n - 1), min_size=m, max_size=m)), dtype=np.int32)
    weighted = draw(st.booleans())
    w = None
    if weighted:
        w = np.array(draw(st.lists(st.floats(0.0009765625, 10.0, allow_nan=False, width=32),
                                   min_size=m, max_size=m)), dtype=np.float32)
    s = np.array(draw(st.lists(st.floats(-2.0, 3.0, allow_nan=False), min_size=n, max_size=n)))
    return n, src, dst, w, s


@hypothesis.settings(max_examples=300, deadline=None, derandomize=True)
@hypothesis.given(graphs())
def test_oracle_routes_and_identities_agree(g):
    n, src, dst, w, s = g
    z_dense = fo.solve_dense(n, src, dst, w, s)
    z_cg = fo.solve_cg(n, src, dst, w, s, tol=1e-13).x
    scale = max(1.0, float(np.max(np.abs(s))))
    assert np.max(np.abs(z_dense - z_cg)) <= 1e-10 * scale

    q = fo.quantities_from_z(n, src, dst, w, s, z_dense)
    forms = fo.quantities_prop1(n, src, dst, w, s)
    norms = fo.quantities_norms(n, src, dst, w, s)
    floor = 1e-12 * max(1.0, float(s @ s))
    for name in fo.QUANTITY_NAMES:
        assert abs(forms[name] - q[name]) <= 1e-9 * abs(q[name]) + floor, (name, forms[name], q[name])
        assert abs(norms[name] - q[name]) <= 1e-9 * abs(q[name]) + floor, (name, norms[name], q[name])

    assert abs(q["I_dc"] - float(s @ z_dense)) <= 1e-9 * abs(q["I_dc"]) + floor
    total = q["C_I"] + 2 * q["D"] + q["C"]
    assert abs(total - float(s @ s)) <= 1e-9 * float(s @ s) + floor
    assert abs(z_dense.sum() - s.sum()) <= 1e-9 * (1.0 + float(np.abs(s).sum()))
    assert z_dense.min() >= s.min() - 1e-12 * scale
    assert z_dense.max() <= s.max() + 1e-12 * scale
