"""Host-side logic of bench.py that needs no GPU: the launch widths and the
byte model behind roofline.achieved, the link between the committed ncu
profile and the kernel sources, and the clock sampler's choice of samples."""
import datetime
import math
import os
import time

import numpy as np
import pytest

import bench


@pytest.mark.parametrize("k", [1, 2, 3, 7, 31, 32, 33, 40, 64, 256, 257])
def test_launch_widths_follow_the_library(k):
    # fj_solve_device runs 32 columns at a time, then the largest power of
    # two that still fits: 16, 8, 4, 2, 1
    widths = bench._launch_widths(k)
    assert sum(widths) == k
    assert widths == sorted(widths, reverse=True)
    assert all(w in (32, 16, 8, 4, 2, 1) for w in widths)
    left = k
    for w in widths:
        assert w == max(v for v in (32, 16, 8, 4, 2, 1) if v <= left)
        left -= w


def test_byte_model_by_hand():
    # n = 10, nnz = 40, weighted, K = 2: graph 4*11 + 40*8 = 364 bytes;
    # 3 iterations of 364 + 52*10*2 and 2 refinements of 364 + 24*10*2
    assert bench._bytes_per_launch(10, 40, True, 2, 3, 2) == 3 * (364 + 1040) + 2 * (364 + 480)
    # unit weights drop the value array
    assert bench._bytes_per_launch(10, 40, False, 1, 1, 0) == 4 * 11 + 40 * 4 + 52 * 10


def test_profile_traffic_only_for_the_profiled_sources(monkeypatch):
    traffic = bench._profiled_traffic()
    assert traffic is None or traffic > 0
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "0" * 64)
    assert bench._profiled_traffic() is None


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


def _sampler(tmp_path, rows, t0, t1):
    path = tmp_path / "clocks.csv"
    fmt = lambda t: datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    with open(path, "w") as f:
        for t, sm, power_cap in rows:
            ts = fmt(t) if t is not None else "n/a"
            cap = "Active" if power_cap else "Not Active"
            f.write(f"{ts}, 0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}\n")
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.proc, c.path, c.device, c.t0, c.t1 = _FakeProc(), str(path), 0, t0, t1
    return c


def test_clock_samples_are_kept_to_the_timed_region(tmp_path):
    now = time.time()
    rows = [(now - 5, 1000, True), (now + 0.1, 2070, False), (now + 0.2, 2060, False), (now + 9, 1200, True)]
    out = _sampler(tmp_path, rows, now, now + 1).stop()
    assert out["window"] == "timed region" and out["samples"] == 2
    assert out["sm_mhz"] == pytest.approx(2065.0) and out["reasons"] == []
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_clock_samples_fall_back_to_the_whole_run(tmp_path):
    now = time.time()
    rows = [(now - 5, 1980, True), (None, 2070, False)]
    out = _sampler(tmp_path, rows, now, now + 1).stop()
    assert out["window"] == "whole run" and out["samples"] == 2
    assert out["reasons"] == ["sw_power_cap"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_quantity_error_bound_holds(seed):
    """The certified sigma bound from a residual: perturb the exact solution,
    and the true relative error of every quantity stays below the bound
    computed from ||s - (I + L) z|| alone (and the bound is not vacuous)."""
    import numpy as np
    import oracle.fj_oracle as fo
    from paper_2101_08143_gb300 import synth
    g = synth.chung_lu(300, 1200, 2.3, seed=seed, weighted=True)
    s = synth.opinions_uniform(g.n, 1, seed)[:, 0]
    z_star = fo.solve_dense(g.n, g.src, g.dst, g.w, s)
    q_star = fo.quantities_from_z(g.n, g.src, g.dst, g.w, s, z_star)
    rng = np.random.default_rng(seed)
    for scale in (1e-9, 1e-6, 1e-4):
        z = z_star + scale * rng.standard_normal(g.n)
        r = s - fo.apply_i_plus_l(g.n, g.src, g.dst, g.w, z)
        eps = float(np.linalg.norm(r))
        q_def = fo.quantities_from_z(g.n, g.src, g.dst, g.w, s, z)
        # a device reduction that is off by a relative 1e-12
        q_gpu = {k: v * (1 + 1e-12) for k, v in q_def.items()}
        bound = bench.quantity_error_bound(q_gpu, q_def, eps)
        for name in fo.QUANTITY_NAMES:
            true_err = abs(q_gpu[name] - q_star[name]) / q_star[name]
            assert true_err <= bound[name], (name, scale, true_err, bound[name])
            assert bound[name] < 1.0


def _stopping_rule_eps(q, t):
    """The largest residual norm the solver's FJ_QUANTITY_TOL rule accepts
    for target t (the device computes the same roots)."""
    tp = t / (1.0 + t)
    best = math.inf
    for name in ("C_I", "D", "P", "C"):
        x = q[name]
        if x > 0:
            a = math.sqrt(x)
            best = min(best, tp * x / (a + math.sqrt(a * a + tp * x)))
    i_dc = q["D"] + q["C"]
    if i_dc > 0:
        b = math.sqrt(q["D"]) + math.sqrt(q["C"])
        best = min(best, tp * i_dc / (b + math.sqrt(b * b + 2.0 * tp * i_dc)))
    return best


def test_stopping_rule_target_inverts_the_certified_bound():
    """At the residual norm the stopping rule accepts, the certified bound
    of the binding quantity equals the target; any larger norm exceeds it."""
    rng = np.random.default_rng(71)
    for _ in range(300):
        q = {name: float(10.0 ** rng.uniform(-3, 8)) for name in ("C_I", "D", "P", "C")}
        q["I_dc"] = q["D"] + q["C"]
        t = float(10.0 ** rng.uniform(-10, -2))
        eps = _stopping_rule_eps(q, t)
        worst = max(bench.quantity_error_bound(q, q, eps).values())
        assert t * (1 - 1e-6) <= worst <= t * (1 + 1e-9), (t, worst)
        assert max(bench.quantity_error_bound(q, q, eps * 1.001).values()) > t
