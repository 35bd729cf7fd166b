"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these checks re-runs the oracle's own formula: each compares it with
a printed value, a closed form, a brute-force enumeration, an independent
route to the same number, or an invariant the paper states.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth


def _read_golden(path):
    rows = []
    meta = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0].isalpha() or "_" in parts[0]:
                meta[parts[0]] = parts[1:]
            else:
                rows.append([int(x) for x in parts])
    return meta, rows


def _random_weighted(n, m, seed, connected=False):
    rng = np.random.default_rng(seed)
    pairs = set()
    if connected:
        for i in range(1, n):
            j = int(rng.integers(0, i))
            pairs.add((j, i))
    while len(pairs) < m:
        a, b = (int(x) for x in rng.integers(0, n, 2))
        if a != b:
            pairs.add((min(a, b), max(a, b)))
    pairs = sorted(pairs)
    src = np.array([p[0] for p in pairs], dtype=np.int32)
    dst = np.array([p[1] for p in pairs], dtype=np.int32)
    w = (0.05 + rng.random(len(pairs)) * 2.0).astype(np.float32)
    return src, dst, w


# ------------------------------------------------------------- Sec. 2.2 pins

def test_p5_forest_matrix_printed(golden_dir):
    """Sec. 2.2 worked example: Omega(P5) = (1/55) [[34, 13, 5, 2, 1], ...]."""
    meta, rows = _read_golden(os.path.join(golden_dir, "p5_forest_matrix.txt"))
    den = int(meta["denominator"][0])
    expect = np.array(rows, dtype=np.float64) / den
    g = synth.path_graph(5)
    om = fo.forest_matrix(5, g.src, g.dst, g.w)
    np.testing.assert_allclose(om, expect, rtol=0, atol=1e-14)
    # The same matrix column by column through both solvers.
    for j in range(5):
        e = np.zeros(5)
        e[j] = 1.0
        np.testing.assert_allclose(fo.solve_dense(5, g.src, g.dst, g.w, e),
                                   expect[:, j], atol=1e-14)
        cg = fo.solve_cg(5, g.src, g.dst, g.w, e, tol=1e-14)
        np.testing.assert_allclose(cg.x, expect[:, j], atol=1e-13)


def _rooted_forest_weights(n, edges):
    """Brute force over all spanning rooted forests (Sec. 2.2): returns
    eps(Gamma) and the matrix eps(Gamma_ij) as exact Fractions, where
    Gamma_ij are the forests with v_i, v_j in one tree rooted at v_i."""
    total = Fraction(0)
    gij = [[Fraction(0)] * n for _ in range(n)]
    m = len(edges)
    for mask in range(1 << m):
        parent = list(range(n))

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x

        weight = Fraction(1)
        acyclic = True
        for e in range(m):
            if mask >> e & 1:
                a, b, wt = edges[e]
                ra, rb = find(a), find(b)
                if ra == rb:
                    acyclic = False
                    break
                parent[ra] = rb
                weight *= wt
        if not acyclic:
            continue
        comp = [find(v) for v in range(n)]
        size = {}
        for c in comp:
            size[c] = size.get(c, 0) + 1
        roots_choices = 1
        for c in size.values():
            roots_choices *= c
        total += weight * roots_choices
        for i in range(n):
            for j in range(n):
                if comp[i] == comp[j]:
                    # tree of v_i has its root fixed to v_i; others free
                    gij[i][j] += weight * roots_choices / size[comp[i]]
    return total, gij


def test_p5_forest_counts():
    """Sec. 2.2: P5 has 55 spanning rooted forests, 13 of them with v2 in a
    tree rooted at v1."""
    edges = [(i, i + 1, Fraction(1)) for i in range(4)]
    total, gij = _rooted_forest_weights(5, edges)
    assert total == 55
    assert gij[0][1] == 13


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forest_matrix_bruteforce_weighted(seed):
    """omega_ij = eps(Gamma_ij) / eps(Gamma) (Sec. 2.2) by enumeration, on
    small weighted graphs, against the oracle's dense and CG solves."""
    n = 5
    src, dst, w = _random_weighted(n, 6, seed)
    edges = [(int(a), int(b), Fraction(float(c))) for a, b, c in
             zip(src, dst, w)]
    total, gij = _rooted_forest_weights(n, edges)
    brute = np.array([[float(gij[i][j] / total) for j in range(n)]
                      for i in range(n)])
    np.testing.assert_allclose(fo.forest_matrix(n, src, dst, w), brute,
                               rtol=1e-13, atol=1e-15)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cg = fo.solve_cg(n, src, dst, w, e, tol=1e-14)
        np.testing.assert_allclose(cg.x, brute[:, j], rtol=1e-11, atol=1e-13)


def test_forest_matrix_disconnected_zero_blocks():
    """omega_ij = 0 exactly when no path joins v_i and v_j (Sec. 2.2)."""
    src = np.array([0, 1, 3], dtype=np.int32)
    dst = np.array([1, 2, 4], dtype=np.int32)
    om = fo.forest_matrix(6, src, dst, None)
    comp = [0, 0, 0, 1, 1, 2]
    for i in range(6):
        for j in range(6):
            if comp[i] != comp[j]:
                assert om[i, j] == 0.0
            else:
                assert om[i, j] > 0.0


@pytest.mark.parametrize("seed", [3, 4])
def test_forest_matrix_spectrum_and_stochastic(seed):
    """Omega is SPD with eigenvalues 1/(1 + lambda_i(L)) and is doubly
    stochastic: Omega 1 = 1, 1^T Omega = 1^T (Sec. 2.2)."""
    n = 40
    src, dst, w = _random_weighted(n, 90, seed)
    om = fo.forest_matrix(n, src, dst, w)
    lam = np.linalg.eigvalsh(fo.laplacian_dense(n, src, dst, w))
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(om)),
                               np.sort(1.0 / (1.0 + lam)), atol=1e-13)
    np.testing.assert_allclose(om.sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(om.sum(axis=0), 1.0, atol=1e-13)
    np.testing.assert_allclose(om, om.T, atol=1e-14)


def test_laplacian_two_constructions():
    """L = D - A equals B^T W B (Sec. 2.1), and the edge-by-edge apply
    matches the dense matrix."""
    n = 30
    src, dst, w = _random_weighted(n, 70, 5)
    L = fo.laplacian_dense(n, src, dst, w)
    B, we = fo.incidence(n, src, dst, w)
    np.testing.assert_allclose(L, B.T @ np.diag(we) @ B, atol=1e-13)
    x = np.random.default_rng(1).random((n, 3))
    np.testing.assert_allclose(fo.apply_laplacian(n, src, dst, w, x), L @ x,
                               atol=1e-12)
    np.testing.assert_allclose(L @ np.ones(n), 0.0, atol=1e-13)


# ---------------------------------------------------- closed forms (Eq. 2)

@pytest.mark.parametrize("n,weight", [(3, None), (17, None), (250, 0.37),
                                      (401, 1.5)])
def test_complete_graph_closed_form(n, weight):
    """K_n with uniform weight w: I + L = (1 + w n) I - w 1 1^T, whose inverse
    (Sherman-Morrison) gives z = (s + w (1^T s) 1) / (1 + w n)."""
    g = synth.complete_graph(n, weight)
    wv = 1.0 if weight is None else float(np.float32(weight))
    s = np.random.default_rng(n).random(n)
    expect = (s + wv * s.sum()) / (1.0 + wv * n)
    z = fo.solve(n, g.src, g.dst, g.w, s)
    np.testing.assert_allclose(z, expect, rtol=1e-11)


def test_k2_hand_worked(golden_dir):
    """Two nodes, one unit edge, s = (1, 0): every quantity by hand."""
    vals = {}
    with open(os.path.join(golden_dir, "k2_hand_values.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, num, den = line.split()
                vals[name] = int(num) / int(den)
    src = np.array([0], np.int32)
    dst = np.array([1], np.int32)
    s = np.array([1.0, 0.0])
    z = fo.solve(2, src, dst, None, s)
    np.testing.assert_allclose(z, [vals["z1"], vals["z2"]], rtol=1e-15)
    q = fo.quantities(2, src, dst, None, s)[0]
    for name in fo.QUANTITY_NAMES:
        assert q[name] == pytest.approx(vals[name], rel=1e-14), name
    a = fo.approxim(2, src, dst, None, s)
    for name in fo.QUANTITY_NAMES:
        assert a[name] == pytest.approx(vals[name], rel=1e-14), name


def test_edgeless_graph():
    """No edges: L = 0, z = s, C_I = D = 0, P = ||s_bar||^2, C = ||s||^2."""
    g = synth.edgeless(300)
    s = np.random.default_rng(2).random(300)
    z = fo.solve(300, g.src, g.dst, g.w, s)
    np.testing.assert_allclose(z, s, rtol=1e-15)
    q = fo.quantities(300, g.src, g.dst, g.w, s)[0]
    assert q["C_I"] == 0.0 and q["D"] == 0.0
    assert q["P"] == pytest.approx(np.sum((s - s.mean()) ** 2), rel=1e-13)
    assert q["C"] == pytest.approx(np.sum(s ** 2), rel=1e-14)


def test_constant_opinions():
    """s = c 1: z = c 1 (Omega 1 = 1), so P = D = C_I = 0, C = n c^2."""
    g = synth.erdos_renyi(500, 2000, seed=3, weighted=True)
    s = np.full(500, 0.3)
    q = fo.quantities(500, g.src, g.dst, g.w, s)[0]
    assert q["C_I"] < 1e-20 and q["D"] < 1e-20 and q["P"] < 1e-20
    assert q["C"] == pytest.approx(500 * 0.09, rel=1e-12)


# ------------------------------------------------ the FJ dynamics (Eq. 1)

def test_fj_update_rule_converges_to_equilibrium():
    """Iterating the update rule (Eq. FJmodel) reaches z = (I+L)^-1 s
    (Eq. FJmodel02)."""
    n = 60
    src, dst, w = _random_weighted(n, 150, 7, connected=True)
    s = np.random.default_rng(0).random(n)
    z_iter = fo.fj_iterate(n, src, dst, w, s, iterations=4000)
    np.testing.assert_allclose(z_iter, fo.solve_dense(n, src, dst, w, s),
                               atol=1e-12)


# --------------------------------------- quantities: three routes, Sec. 3-4

@pytest.mark.parametrize("seed,connected", [(11, True), (12, False),
                                            (13, True)])
def test_quantity_routes_agree(seed, connected):
    """Definitions (Sec. 3.2) == Proposition 1 quadratic forms == Lemma PropA
    norms == Algorithm 1, on small weighted graphs."""
    n = 120
    src, dst, w = _random_weighted(n, 300, seed, connected)
    s = np.random.default_rng(seed).random(n)
    ref = fo.quantities(n, src, dst, w, s)[0]
    for other in (fo.quantities_prop1(n, src, dst, w, s),
                  fo.quantities_norms(n, src, dst, w, s),
                  fo.approxim(n, src, dst, w, s)):
        for name in fo.QUANTITY_NAMES:
            assert other[name] == pytest.approx(ref[name], rel=1e-11), name


def _identities(n, src, dst, w, s, q, rtol):
    z = fo.solve(n, src, dst, w, s)
    # I_dc = D + C = s^T z (Sec. 3.2, after the definition of I_dc)
    assert q["I_dc"] == pytest.approx(float(s @ z), rel=rtol)
    # s - z = L z gives C_I + D = s^T s - s^T z, hence C_I + 2D + C = ||s||^2
    assert q["C_I"] + 2 * q["D"] + q["C"] == pytest.approx(float(s @ s),
                                                           rel=rtol)
    # 1^T z = 1^T s (Sec. 3.1 conservation) gives P = C - (1^T s)^2 / n
    assert q["P"] == pytest.approx(q["C"] - s.sum() ** 2 / n, rel=1e3 * rtol)
    # Conservation of the total opinion (Sec. 3.1)
    assert z.sum() == pytest.approx(s.sum(), rel=rtol)
    # z_i lies within the range of s (Omega is doubly stochastic, >= 0)
    assert z.min() >= s.min() - 1e-12 and z.max() <= s.max() + 1e-12


def test_identities_erdos_renyi_cg_mode():
    """n = 2000 ER graph (above the dense limit, so the CG path)."""
    g = synth.erdos_renyi(2000, 10000, seed=1)
    s = synth.opinions_uniform(2000, 1, 1001)[:, 0]
    q = fo.quantities(2000, g.src, g.dst, g.w, s)[0]
    _identities(2000, g.src, g.dst, g.w, s, q, 1e-10)


def test_identities_chung_lu_weighted():
    g = synth.chung_lu(20_000, 60_000, 2.3, seed=9, weighted=True)
    s = synth.opinions_polarized(g.n, 1, 5)[:, 0]
    q = fo.quantities(g.n, g.src, g.dst, g.w, s)[0]
    _identities(g.n, g.src, g.dst, g.w, s, q, 1e-9)


@pytest.mark.parametrize("seed", [21, 22])
def test_cg_matches_dense(seed):
    n = 180
    src, dst, w = _random_weighted(n, 500, seed)
    s = np.random.default_rng(seed).random(n)
    cg = fo.solve_cg(n, src, dst, w, s, tol=1e-13)
    assert cg.rel_residual <= 1e-13
    np.testing.assert_allclose(cg.x, fo.solve_dense(n, src, dst, w, s),
                               rtol=1e-11)


def test_parallel_edges_add_and_self_loops_vanish():
    """A repeated pair acts as one edge of the summed weight; a self-loop
    adds nothing to L (b_e = 0), Sec. 2.1."""
    src = np.array([0, 1, 0, 2, 2], np.int32)
    dst = np.array([1, 2, 1, 2, 3], np.int32)
    w = np.array([0.5, 1.0, 0.25, 9.0, 2.0], np.float32)
    s = np.array([0.9, 0.1, 0.4, 0.7])
    merged = fo.solve_dense(4, np.array([0, 1, 2]), np.array([1, 2, 3]),
                            np.array([0.75, 1.0, 2.0], np.float32), s)
    np.testing.assert_allclose(fo.solve_dense(4, src, dst, w, s), merged,
                               rtol=1e-15)
    np.testing.assert_allclose(fo.solve_cg(4, src, dst, w, s, 1e-14).x,
                               merged, rtol=1e-13)


def test_residual_rows_matches_full_residual():
    g = synth.chung_lu(3000, 9000, 2.3, seed=4, weighted=True)
    s = np.random.default_rng(1).random(g.n)
    z = np.random.default_rng(2).random(g.n)
    full = s - fo.apply_i_plus_l(g.n, g.src, g.dst, g.w, z)
    rows = np.array([0, 5, 17, 2999, 1234])
    np.testing.assert_allclose(
        fo.residual_rows(g.n, g.src, g.dst, g.w, z, s, rows), full[rows],
        atol=1e-12)


def test_relative_error_metric():
    assert fo.relative_error(2.0, 2.002) == pytest.approx(1e-3)
    assert fo.relative_error(0.0, 1e-15, floor=1e-12) == pytest.approx(1e-3)


# ------------------------------------ planted mistakes are caught by pins

def test_planted_mistakes_are_caught(monkeypatch):
    """Plant typical slips in the oracle (CPU only) and check that the pins
    above reject each of them."""
    g = synth.erdos_renyi(250, 900, seed=6, weighted=True)
    s = np.random.default_rng(3).random(250)

    def pins_pass():
        try:
            q = fo.quantities(250, g.src, g.dst, g.w, s)[0]
            _identities(250, g.src, g.dst, g.w, s, q, 1e-10)
            other = fo.quantities_norms(250, g.src, g.dst, g.w, s)
            for name in fo.QUANTITY_NAMES:
                assert other[name] == pytest.approx(q[name], rel=1e-10)
            return True
        except AssertionError:
            return False

    assert pins_pass()
    orig_from_z = fo.quantities_from_z

    def drop_weight(n, src, dst, w, s_, z):  # D without w_ij
        q = orig_from_z(n, src, dst, None, s_, z)
        return q

    monkeypatch.setattr(fo, "quantities_from_z", drop_weight)
    assert not pins_pass()
    monkeypatch.undo()

    orig_lap = fo.laplacian_dense

    def transposed_sign(n, src, dst, w):  # A + D instead of D - A
        L = orig_lap(n, src, dst, w)
        return 2 * np.diag(np.diag(L)) - L

    monkeypatch.setattr(fo, "laplacian_dense", transposed_sign)
    assert not pins_pass()
    monkeypatch.undo()

    def mean_not_removed(s_):  # s_bar = s
        return np.asarray(s_, dtype=np.float64)

    monkeypatch.setattr(fo, "centred", mean_not_removed)
    assert not pins_pass()
    monkeypatch.undo()
    assert pins_pass()


def _planted(name):
    """A plausible slip in the oracle, as a (function name, replacement)
    pair for monkeypatching."""
    orig_apply = fo.apply_laplacian
    orig_from_z = fo.quantities_from_z
    if name == "weights squared in L x":
        return "apply_laplacian", lambda n, src, dst, w, x: orig_apply(
            n, src, dst, None if w is None else np.asarray(w, dtype=np.float64) ** 2, x)
    if name == "weights of the wrong edges in L x":
        return "apply_laplacian", lambda n, src, dst, w, x: orig_apply(
            n, src, dst, None if w is None else np.asarray(w)[::-1].copy(), x)
    if name == "D over both directions":
        def f(n, src, dst, w, s_, z):
            q = dict(orig_from_z(n, src, dst, w, s_, z))
            q["D"] *= 2
            q["I_dc"] = q["D"] + q["C"]
            return q
        return "quantities_from_z", f
    if name == "C_I against s_bar":
        def f(n, src, dst, w, s_, z):
            q = dict(orig_from_z(n, src, dst, w, s_, z))
            q["C_I"] = float(np.sum((np.asarray(z) - fo.centred(s_)) ** 2))
            return q
        return "quantities_from_z", f
    if name == "P without centring z":
        def f(n, src, dst, w, s_, z):
            q = dict(orig_from_z(n, src, dst, w, s_, z))
            q["P"] = q["C"]
            return q
        return "quantities_from_z", f
    raise KeyError(name)


@pytest.mark.parametrize("name", ["weights squared in L x", "weights of the wrong edges in L x",
                                  "D over both directions", "C_I against s_bar",
                                  "P without centring z"])
def test_more_planted_mistakes_are_caught(monkeypatch, name):
    """Further slips, each planted in the CG path (n = 250 > the dense limit)
    or in the definitions: the identities or the dense Lemma PropA norms
    reject every one."""
    g = synth.erdos_renyi(250, 900, seed=6, weighted=True)
    s = np.random.default_rng(3).random(250)

    def pins_pass():
        try:
            q = fo.quantities(250, g.src, g.dst, g.w, s)[0]
            _identities(250, g.src, g.dst, g.w, s, q, 1e-10)
            other = fo.quantities_norms(250, g.src, g.dst, g.w, s)
            for qn in fo.QUANTITY_NAMES:
                assert other[qn] == pytest.approx(q[qn], rel=1e-10)
            return True
        except AssertionError:
            return False

    assert pins_pass()
    attr, repl = _planted(name)
    monkeypatch.setattr(fo, attr, repl)
    assert not pins_pass()
    monkeypatch.undo()
    assert pins_pass()


# ------------------------------------------------- largest connected component

def _bfs_components(n, src, dst):
    adj = [[] for _ in range(n)]
    for a, b in zip(src, dst):
        if a != b:
            adj[a].append(b)
            adj[b].append(a)
    comp = [-1] * n
    comps = []
    for v in range(n):
        if comp[v] >= 0:
            continue
        comp[v] = len(comps)
        stack, members = [v], [v]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if comp[y] < 0:
                    comp[y] = comp[v]
                    stack.append(y)
                    members.append(y)
        comps.append(sorted(members))
    return comps


@pytest.mark.parametrize("seed", range(6))
def test_largest_component_matches_breadth_first_search(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    m = int(rng.integers(0, 2 * n))
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    w = rng.uniform(0.1, 1.0, m).astype(np.float32)
    comps = _bfs_components(n, src, dst)
    want = max(comps, key=lambda c: (len(c), -c[0]))
    nodes, s2, d2, w2 = fo.largest_component(n, src, dst, w)
    assert list(nodes) == want
    pos = {v: i for i, v in enumerate(want)}
    exp = sorted((pos[a], pos[b], float(x)) for a, b, x in zip(src, dst, w)
                 if a != b and a in pos)
    assert sorted(zip(s2.tolist(), d2.tolist(), w2.tolist())) == exp


def test_largest_component_ties_go_to_the_smallest_id():
    # two triangles {1,2,3} and {0,4,5}, one isolated node 6
    src = np.array([1, 2, 3, 4, 5, 0])
    dst = np.array([2, 3, 1, 5, 0, 4])
    nodes, s2, d2, _ = fo.largest_component(7, src, dst, None)
    assert list(nodes) == [0, 4, 5]
    assert sorted(zip(s2, d2)) == [(0, 1), (1, 2), (2, 0)]
