"""Seeded synthetic inputs: graphs and innate-opinion vectors.

This module is the one piece shared by the CUDA path's tests/bench and the CPU
oracle.  It holds no arithmetic of the method itself (no Laplacian, no solve,
no quantity): it only draws edge lists and opinion vectors from seeded numpy
generators (PCG64), whose streams are the same on every platform.  The one
floating-point step before a draw, the Chung-Lu CDF, could differ by an ulp
between math libraries, which changes a draw only if a variate falls inside
that ulp; each test and the benchmark generate their inputs on the machine
that runs them.

Graph model (Sec. 2.1 of the paper): undirected, simple, weighted, w_e > 0.
Generators emit simple graphs (no self-loops, no duplicate pairs).

* Erdos-Renyi G(n, m): pairs drawn uniformly, deduplicated until at least m
  distinct pairs exist, then m of them kept at random.
* Chung-Lu power law: node weights (i+1)^(-1/(beta-1)); both endpoints drawn
  proportionally to them (inverse CDF through a guide table); self-loops and
  repeated pairs dropped; drawing is repeated until at least m distinct edges
  exist and m of them are kept at random; node ids are then permuted at
  random so that hubs are not simply the lowest ids.
* Edge weights: 1.0 (unit) or Uniform(0, 1] rounded to float32.  The float32
  values are the ground truth both sides read.
* Opinions (Sec. 5, "Internal opinion distributions"): Uniform[0,1]; the
  polarized Beta(0.5, 0.5) mix (sin^2(pi U / 2)); and the paper's exponential
  and power-law (alpha = 2.5) draws normalised by their maximum.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class EdgeList:
    """An undirected weighted edge list (each undirected edge listed once)."""

    n: int
    src: np.ndarray  # int32 [m]
    dst: np.ndarray  # int32 [m]
    w: np.ndarray | None  # float32 [m], or None for unit weights

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def weights_f64(self) -> np.ndarray:
        if self.w is None:
            return np.ones(self.m, dtype=np.float64)
        return self.w.astype(np.float64)


def _distinct_keys(u: np.ndarray, v: np.ndarray, n: int) -> np.ndarray:
    """Sorted distinct keys lo * n + hi of the unordered pairs {u, v}, with
    self-loops dropped."""
    keep = u != v
    lo = np.minimum(u[keep], v[keep]).astype(np.int64)
    hi = np.maximum(u[keep], v[keep]).astype(np.int64)
    key = lo * n + hi
    key.sort()
    if key.shape[0] == 0:
        return key
    first = np.empty(key.shape[0], dtype=bool)
    first[0] = True
    np.not_equal(key[1:], key[:-1], out=first[1:])
    return key[first]


def _collect_edges(draw, n: int, m: int, rng: np.random.Generator):
    """Draw candidate pairs with `draw(count)` until m distinct unordered pairs
    exist, then keep m of them chosen uniformly at random, in random order
    (each as (lower id, higher id))."""
    keys = np.empty(0, dtype=np.int64)
    factor = 1.25
    while keys.shape[0] < m:
        need = m - keys.shape[0]
        cnt = max(1024, int(need * factor))
        u, v = draw(cnt)
        new = _distinct_keys(u, v, n)
        keys = new if keys.shape[0] == 0 else np.union1d(keys, new)
        factor *= 1.5
    keys = keys[rng.permutation(keys.shape[0])[:m]]
    return keys // n, keys % n


def _inverse_cdf(cdf: np.ndarray, guide: np.ndarray, r: np.ndarray) -> np.ndarray:
    """For each r in [0, 1): the smallest i with cdf[i] > r (what
    np.searchsorted(cdf, r, side="right") returns), found from a guide table
    (Chen and Asau, 1974): guide[b] is that index for r = b / len(guide), so
    the search starts at most one bucket early and steps forward."""
    M = guide.shape[0]
    b = np.floor(r * M).astype(np.int64) - 1
    np.clip(b, 0, M - 1, out=b)
    i = guide[b]
    last = cdf.shape[0] - 1
    idx = np.nonzero(cdf[i] <= r)[0]
    while idx.shape[0]:
        i[idx] += 1
        np.minimum(i, last, out=i)
        idx = idx[(cdf[i[idx]] <= r[idx]) & (i[idx] < last)]
    return i


def _weights(rng: np.random.Generator, m: int, weighted: bool):
    if not weighted:
        return None
    # Uniform(0, 1]: 1 - U[0,1) never hits 0; float32 rounding keeps it > 0
    # (the smallest value 2^-53 is a normal float32).
    return (1.0 - rng.random(m)).astype(np.float32)


def erdos_renyi(n: int, m: int, seed: int, weighted: bool = False) -> EdgeList:
    """G(n, m): m distinct uniformly random unordered pairs, no self-loops."""
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the number of node pairs")
    rng = np.random.default_rng(seed)

    def draw(cnt):
        return (rng.integers(0, n, cnt, dtype=np.int64),
                rng.integers(0, n, cnt, dtype=np.int64))

    u, v = _collect_edges(draw, n, m, rng)
    w = _weights(rng, m, weighted)
    return EdgeList(n, u.astype(np.int32), v.astype(np.int32), w)


def chung_lu(n: int, m: int, exponent: float, seed: int,
             weighted: bool = False) -> EdgeList:
    """Chung-Lu power-law graph with expected degrees proportional to
    (i+1)^(-1/(exponent-1)), m distinct edges, ids randomly permuted."""
    rng = np.random.default_rng(seed)
    a = 1.0 / (exponent - 1.0)
    cdf = np.cumsum((np.arange(n, dtype=np.float64) + 1.0) ** (-a))
    cdf /= cdf[-1]

    guide = np.searchsorted(cdf, np.arange(2 * n, dtype=np.float64) / (2 * n), side="right")
    np.minimum(guide, n - 1, out=guide)

    def draw(cnt):
        u = _inverse_cdf(cdf, guide, rng.random(cnt))
        v = _inverse_cdf(cdf, guide, rng.random(cnt))
        return u, v

    u, v = _collect_edges(draw, n, m, rng)
    perm = rng.permutation(n).astype(np.int64)
    u, v = perm[u], perm[v]
    w = _weights(rng, m, weighted)
    return EdgeList(n, u.astype(np.int32), v.astype(np.int32), w)


def path_graph(n: int) -> EdgeList:
    """Unit-weight path v1 - v2 - ... - vn."""
    src = np.arange(n - 1, dtype=np.int32)
    return EdgeList(n, src, src + 1, None)


def complete_graph(n: int, weight: float | None = None) -> EdgeList:
    """K_n with every edge of the given weight (None: unit)."""
    iu, ju = np.triu_indices(n, 1)
    w = None if weight is None else np.full(iu.shape[0], weight, np.float32)
    return EdgeList(n, iu.astype(np.int32), ju.astype(np.int32), w)


def edgeless(n: int) -> EdgeList:
    e = np.empty(0, dtype=np.int32)
    return EdgeList(n, e, e.copy(), None)


# ----------------------------------------------------------------- opinions

def opinions_uniform(n: int, k: int, seed: int) -> np.ndarray:
    """s ~ Uniform[0,1], float64, column-major n x k (Fortran order)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.random((k, n)).T)


def opinions_polarized(n: int, k: int, seed: int) -> np.ndarray:
    """Beta(0.5, 0.5) opinions, drawn as sin^2(pi U / 2); n x k column-major."""
    rng = np.random.default_rng(seed)
    u = rng.random((k, n)).T
    return np.asfortranarray(np.sin(0.5 * math.pi * u) ** 2)


def opinions_batch_mix(n: int, k: int, seed: int) -> np.ndarray:
    """First half of the columns Uniform[0,1], second half Beta(0.5, 0.5)."""
    h = k // 2
    a = opinions_uniform(n, k - h, seed)
    b = opinions_polarized(n, h, seed + 7919)
    return np.asfortranarray(np.concatenate([a, b], axis=1))


def opinions_exponential(n: int, k: int, seed: int, x_min: float = 1.0):
    """Density e^{x_min} e^{-x} on x >= x_min, divided by the column max."""
    rng = np.random.default_rng(seed)
    x = x_min + rng.exponential(1.0, (k, n)).T
    return np.asfortranarray(x / x.max(axis=0, keepdims=True))


def opinions_power_law(n: int, k: int, seed: int, alpha: float = 2.5,
                       x_min: float = 1.0):
    """Density (alpha-1) x_min^(alpha-1) x^-alpha, divided by the column max."""
    rng = np.random.default_rng(seed)
    u = rng.random((k, n)).T
    x = x_min * (1.0 - u) ** (-1.0 / (alpha - 1.0))
    return np.asfortranarray(x / x.max(axis=0, keepdims=True))


# ------------------------------------------------------- named workloads

WORKLOADS = {
    # name: (generator, kwargs, k, opinion sampler, seed)
    "er_n2k_d10": dict(kind="er", n=2_000, m=10_000, weighted=False, k=1,
                       opinions="uniform", seed=1),
    "cl_n1m_m5m_b2.3": dict(kind="cl", n=1_000_000, m=5_000_000,
                            exponent=2.3, weighted=True, k=1,
                            opinions="uniform", seed=2),
    "cl_n4m_m40m_b2.1_k256": dict(kind="cl", n=4_000_000, m=40_000_000,
                                  exponent=2.1, weighted=False, k=256,
                                  opinions="mix", seed=3),
    "cl_n20m_m150m_b2.1": dict(kind="cl", n=20_000_000, m=150_000_000,
                               exponent=2.1, weighted=True, k=1,
                               opinions="uniform", seed=5),
    # the 20M/150M shape scaled down five-fold (profiling captures)
    "cl_n4m_m30m_b2.1": dict(kind="cl", n=4_000_000, m=30_000_000,
                             exponent=2.1, weighted=True, k=1,
                             opinions="uniform", seed=6),
}


def make_graph(spec: dict) -> EdgeList:
    if spec["kind"] == "er":
        return erdos_renyi(spec["n"], spec["m"], spec["seed"],
                           spec.get("weighted", False))
    return chung_lu(spec["n"], spec["m"], spec["exponent"], spec["seed"],
                    spec.get("weighted", False))


def make_opinions(spec: dict, n: int, k: int | None = None) -> np.ndarray:
    k = spec["k"] if k is None else k
    seed = spec["seed"] + 1000
    kind = spec.get("opinions", "uniform")
    if kind == "uniform":
        return opinions_uniform(n, k, seed)
    if kind == "mix":
        return opinions_batch_mix(n, k, seed)
    if kind == "polarized":
        return opinions_polarized(n, k, seed)
    if kind == "exponential":
        return opinions_exponential(n, k, seed)
    if kind == "power_law":
        return opinions_power_law(n, k, seed)
    raise ValueError(kind)
