"""FP64 CPU oracle for the Friedkin-Johnsen quantities (Xu, Bao, Zhang,
"Fast Evaluation for Relevant Quantities of Opinion Dynamics", WWW 2021).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module.  The CUDA library never
calls it and shares no code with it; the only thing both sides read is the
seeded input (edge lists and opinion vectors).

Everything here is plain, single-threaded numpy in float64, written so that it
can be checked against the paper by eye:

* the graph model of Sec. 2.1 (adjacency A, weighted degrees d, D, L = D - A,
  and the incidence form L = B^T W B = sum_e w_e b_e b_e^T);
* the forest matrix Omega = (I + L)^-1 of Sec. 2.2;
* the FJ update rule (Eq. FJmodel) and its equilibrium z = (I + L)^-1 s
  (Eq. FJmodel02, Sec. 3.1);
* the five quantities by their definitions in Sec. 3.2 (internal conflict,
  disagreement, polarization, controversy, disagreement-controversy index),
  their quadratic forms (Proposition 1) and their l2-norm forms (Lemma PropA);
* Algorithm 1 (APPROXIM) step by step, with Solve() realised by an FP64
  conjugate-gradient solve;
* the subgraph induced on the largest connected component, on which the
  paper's experiments run (Sec. 5), with scipy's connected_components as the
  component step.

Readings of the paper used here (where it is silent or garbled):

* Edge weights arrive as float32 and are upcast exactly; a missing weight
  array means unit weights (the paper's conclusion says "unweighted", Sec. 2.1
  says weighted: unit weights are the special case).
* Self-loops are dropped (b_e = e_i - e_i = 0 adds nothing to L); a repeated
  pair is a parallel edge whose weights add, which is what L = sum_e w_e b_e
  b_e^T gives.
* Connectivity is not required: I + L is positive definite for every graph.
* Algorithm 1 computes delta from ||s_bar|| before s_bar is formed; here s_bar
  comes first.  The literal delta (about 1e-31 at n = 1e6) is below float64
  resolution, so Solve() runs CG to a relative residual `tol` instead.
"""
from __future__ import annotations

import dataclasses

import numpy as np

DENSE_MAX_N = 200

QUANTITY_NAMES = ("C_I", "D", "P", "C", "I_dc")


# ---------------------------------------------------------------- the graph

def clean_edges(n, src, dst, w):
    """Edge arrays in float64 with self-loops removed (Sec. 2.1: simple graph,
    weights w_e > 0).  Raises on out-of-range ids or non-positive weights."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if w is None:
        w = np.ones(src.shape[0], dtype=np.float64)
    else:
        w = np.asarray(w).astype(np.float64)
    if src.shape != dst.shape or src.shape != w.shape:
        raise ValueError("src, dst, w must have one entry per edge")
    if src.size and (src.min() < 0 or dst.min() < 0 or
                     src.max() >= n or dst.max() >= n):
        raise ValueError("node id out of range")
    if src.size and not (np.all(np.isfinite(w)) and np.all(w > 0)):
        raise ValueError("edge weights must be finite and > 0")
    keep = src != dst
    return src[keep], dst[keep], w[keep]


def adjacency_dense(n, src, dst, w):
    """A = (w_ij), symmetric, Sec. 2.1."""
    src, dst, w = clean_edges(n, src, dst, w)
    A = np.zeros((n, n), dtype=np.float64)
    np.add.at(A, (src, dst), w)
    np.add.at(A, (dst, src), w)
    return A


def laplacian_dense(n, src, dst, w):
    """L = D - A with D = diag(d), d_i = sum_j w_ij (Sec. 2.1)."""
    A = adjacency_dense(n, src, dst, w)
    return np.diag(A.sum(axis=1)) - A


def incidence(n, src, dst, w):
    """Signed edge-node incidence B (m x n), b_e = e_head - e_tail, and the
    edge weights (the diagonal of W), Sec. 2.1."""
    src, dst, w = clean_edges(n, src, dst, w)
    m = src.shape[0]
    B = np.zeros((m, n), dtype=np.float64)
    B[np.arange(m), src] = 1.0
    B[np.arange(m), dst] = -1.0
    return B, w


def weighted_degrees(n, src, dst, w):
    """d_i = sum over edges at i of w_e (Sec. 2.1)."""
    src, dst, w = clean_edges(n, src, dst, w)
    return (np.bincount(src, weights=w, minlength=n) +
            np.bincount(dst, weights=w, minlength=n))


def apply_laplacian(n, src, dst, w, x):
    """L x = sum_e w_e b_e (b_e^T x), the incidence form of Sec. 2.1, applied
    edge by edge; x may be a vector or an n x k array."""
    src, dst, w = clean_edges(n, src, dst, w)
    x = np.asarray(x, dtype=np.float64)
    cols = x.reshape(n, -1)
    out = np.empty_like(cols)
    for c in range(cols.shape[1]):
        diff = w * (cols[src, c] - cols[dst, c])  # w_e * (b_e^T x)
        out[:, c] = (np.bincount(src, weights=diff, minlength=n) -
                     np.bincount(dst, weights=diff, minlength=n))
    return out.reshape(x.shape)


def apply_i_plus_l(n, src, dst, w, x):
    """(I + L) x."""
    return np.asarray(x, dtype=np.float64) + apply_laplacian(n, src, dst, w, x)


def largest_component(n, src, dst, w):
    """The subgraph induced on the largest connected component (the paper's
    experiments run on each network's largest connected component, Sec. 5):
    its nodes in increasing id, and its edges (self-loops dropped) renumbered
    to positions in that list, with their weights.  Of components of equal
    size, the one holding the smallest node id wins.  Components come from
    scipy's connected_components."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    src, dst, w = clean_edges(n, src, dst, w)
    adj = coo_matrix((np.ones(src.shape[0]), (src, dst)), shape=(n, n))
    ncomp, labels = connected_components(adj, directed=False)
    sizes = np.bincount(labels, minlength=ncomp)
    min_id = np.full(ncomp, n, dtype=np.int64)
    np.minimum.at(min_id, labels, np.arange(n))
    best = max(range(ncomp), key=lambda c: (sizes[c], -min_id[c]))
    nodes = np.nonzero(labels == best)[0]
    new = np.full(n, -1, dtype=np.int64)
    new[nodes] = np.arange(nodes.shape[0])
    keep = labels[src] == best
    return nodes, new[src[keep]], new[dst[keep]], w[keep]


# ------------------------------------------------------- the linear system

def forest_matrix(n, src, dst, w):
    """Omega = (I + L)^-1 formed densely (Sec. 2.2); small n only."""
    M = np.eye(n) + laplacian_dense(n, src, dst, w)
    return np.linalg.inv(M)


def solve_dense(n, src, dst, w, s):
    """z = (I + L)^-1 s by a dense LU solve (Eq. FJmodel02)."""
    M = np.eye(n) + laplacian_dense(n, src, dst, w)
    return np.linalg.solve(M, np.asarray(s, dtype=np.float64))


@dataclasses.dataclass
class CGResult:
    x: np.ndarray
    iterations: int
    rel_residual: float


def solve_cg(n, src, dst, w, b, tol=1e-12, max_iter=100_000):
    """Solve (I + L) x = b for one right-hand side with Jacobi-preconditioned
    conjugate gradients (Hestenes-Stiefel form), in float64.

    Preconditioner M = diag(1 + d_i).  Stops when ||b - (I+L)x|| <= tol ||b||,
    the residual being recomputed from scratch at the end.
    """
    b = np.asarray(b, dtype=np.float64)
    src, dst, w = clean_edges(n, src, dst, w)
    minv = 1.0 / (1.0 + weighted_degrees(n, src, dst, w))
    bnorm = float(np.sqrt(np.dot(b, b)))
    x = np.zeros(n)
    if bnorm == 0.0:
        return CGResult(x, 0, 0.0)
    r = b.copy()
    zt = minv * r
    p = zt.copy()
    rz = float(np.dot(r, zt))
    it = 0
    while it < max_iter:
        if np.sqrt(np.dot(r, r)) <= tol * bnorm:
            break
        Ap = apply_i_plus_l(n, src, dst, w, p)
        alpha = rz / float(np.dot(p, Ap))
        x += alpha * p
        r -= alpha * Ap
        zt = minv * r
        rz_new = float(np.dot(r, zt))
        p = zt + (rz_new / rz) * p
        rz = rz_new
        it += 1
    true_r = b - apply_i_plus_l(n, src, dst, w, x)
    return CGResult(x, it, float(np.sqrt(np.dot(true_r, true_r)) / bnorm))


def solve(n, src, dst, w, s, tol=1e-12):
    """z = (I + L)^-1 s: dense for n <= 200, FP64 CG above.  s may be n x k."""
    s = np.asarray(s, dtype=np.float64)
    if n <= DENSE_MAX_N:
        return solve_dense(n, src, dst, w, s)
    if s.ndim == 1:
        return solve_cg(n, src, dst, w, s, tol).x
    out = np.empty_like(s, order="F")
    for c in range(s.shape[1]):
        out[:, c] = solve_cg(n, src, dst, w, s[:, c], tol).x
    return out


def fj_iterate(n, src, dst, w, s, iterations):
    """The FJ update rule (Eq. FJmodel) applied synchronously to all nodes,
    starting from z = s:  z_i <- (s_i + sum_j w_ij z_j) / (1 + sum_j w_ij)."""
    src, dst, w = clean_edges(n, src, dst, w)
    s = np.asarray(s, dtype=np.float64)
    d = weighted_degrees(n, src, dst, w)
    z = s.copy()
    for _ in range(iterations):
        az = (np.bincount(src, weights=w * z[dst], minlength=n) +
              np.bincount(dst, weights=w * z[src], minlength=n))
        z = (s + az) / (1.0 + d)
    return z


# -------------------------------------------------------------- quantities

def centred(s):
    """s_bar = s - (1^T s / n) 1 (Sec. 3.2, before Proposition 1)."""
    s = np.asarray(s, dtype=np.float64)
    return s - s.mean(axis=0)


def quantities_from_z(n, src, dst, w, s, z):
    """The five quantities by their definitions (Sec. 3.2), for one opinion
    vector s and its equilibrium z:

      C_I  = sum_i (z_i - s_i)^2                      (internal conflict)
      D    = sum_{(i,j) in E} w_ij (z_i - z_j)^2      (disagreement)
      P    = sum_i (z_i - zbar)^2, zbar = z^T 1 / n   (polarization)
      C    = sum_i z_i^2                              (controversy)
      I_dc = D + C                                    (disagreement-controversy)
    """
    src, dst, w = clean_edges(n, src, dst, w)
    s = np.asarray(s, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    c_i = float(np.sum((z - s) ** 2))
    dis = float(np.sum(w * (z[src] - z[dst]) ** 2))
    zc = z - np.sum(z) / n
    pol = float(np.sum(zc ** 2))
    con = float(np.sum(z ** 2))
    return {"C_I": c_i, "D": dis, "P": pol, "C": con, "I_dc": dis + con}


def quantities(n, src, dst, w, s, tol=1e-12):
    """Five quantities of every column of s (n or n x k): solve, then apply
    the definitions.  Returns a list of dicts, one per column."""
    s = np.asarray(s, dtype=np.float64)
    cols = s.reshape(n, -1)
    z = solve(n, src, dst, w, cols, tol)
    z = z.reshape(n, -1)
    return [quantities_from_z(n, src, dst, w, cols[:, c], z[:, c])
            for c in range(cols.shape[1])]


def quantities_prop1(n, src, dst, w, s):
    """Proposition 1: the quantities as quadratic forms in s through the
    dense forest matrix Omega = (I+L)^-1 (small n only)."""
    s = np.asarray(s, dtype=np.float64)
    L = laplacian_dense(n, src, dst, w)
    Om = np.linalg.inv(np.eye(n) + L)
    sb = centred(s)
    c_i = s @ Om @ L @ L @ Om @ s
    dis = s @ Om @ L @ Om @ s
    pol = sb @ Om @ Om @ sb
    con = s @ Om @ Om @ s
    idc = s @ Om @ s
    return {"C_I": float(c_i), "D": float(dis), "P": float(pol),
            "C": float(con), "I_dc": float(idc)}


def quantities_norms(n, src, dst, w, s):
    """Lemma PropA: the quantities as squared l2 norms (small n only):
    C_I = ||L Om s||^2, D = ||W^1/2 B Om s||^2, P = ||Om s_bar||^2,
    C = ||Om s||^2, I_dc = D + C."""
    s = np.asarray(s, dtype=np.float64)
    L = laplacian_dense(n, src, dst, w)
    B, we = incidence(n, src, dst, w)
    Om = np.linalg.inv(np.eye(n) + L)
    z = Om @ s
    dvec = np.sqrt(we) * (B @ z)
    return {"C_I": float(np.sum((L @ z) ** 2)),
            "D": float(np.sum(dvec ** 2)),
            "P": float(np.sum((Om @ centred(s)) ** 2)),
            "C": float(np.sum(z ** 2)),
            "I_dc": float(np.sum(dvec ** 2) + np.sum(z ** 2))}


def approxim(n, src, dst, w, s, tol=1e-12):
    """Algorithm 1 (APPROXIM) in the paper's order and notation, with
    Solve(I+L, x, delta) realised by FP64 CG to relative residual `tol`:

      s_bar = s - (1^T s / n) 1
      z~    = Solve(I + L, s)         q = Solve(I + L, s_bar)
      C_I   = ||L z~||^2              D = ||W^1/2 B q||^2
      P     = ||q||^2                 C = ||z~||^2
      I_dc  = D + C
    """
    s = np.asarray(s, dtype=np.float64)
    src, dst, w = clean_edges(n, src, dst, w)
    s_bar = centred(s)
    if n <= DENSE_MAX_N:
        z_t = solve_dense(n, src, dst, w, s)
        q = solve_dense(n, src, dst, w, s_bar)
    else:
        z_t = solve_cg(n, src, dst, w, s, tol).x
        q = solve_cg(n, src, dst, w, s_bar, tol).x
    lz = apply_laplacian(n, src, dst, w, z_t)
    wb_q = np.sqrt(w) * (q[src] - q[dst])  # W^1/2 B q, one entry per edge
    dis = float(np.sum(wb_q ** 2))
    con = float(np.sum(z_t ** 2))
    return {"C_I": float(np.sum(lz ** 2)), "D": dis,
            "P": float(np.sum(q ** 2)), "C": con, "I_dc": dis + con}


# ------------------------------------------------------------- error metric

def relative_error(exact, approx, floor=0.0):
    """sigma = |rho - rho~| / rho (Sec. 5, Accuracy), with a floor for
    quantities that are zero (constant opinions, edgeless graphs)."""
    return abs(approx - exact) / max(abs(exact), floor)


def residual_rows(n, src, dst, w, z, s, rows):
    """(s - (I + L) z)_i for selected rows i only, from the edge list: lets a
    caller check a solution of a graph too large to solve here."""
    src, dst, w = clean_edges(n, src, dst, w)
    rows = np.asarray(rows, dtype=np.int64)
    z = np.asarray(z, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    sel = np.zeros(n, dtype=bool)
    sel[rows] = True
    out = np.zeros(n)
    m_src = sel[src]
    m_dst = sel[dst]
    d1 = w[m_src] * (z[src[m_src]] - z[dst[m_src]])
    d2 = w[m_dst] * (z[dst[m_dst]] - z[src[m_dst]])
    np.add.at(out, src[m_src], d1)
    np.add.at(out, dst[m_dst], d2)
    return s[rows] - z[rows] - out[rows]
