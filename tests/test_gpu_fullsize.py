"""Parity at the full sizes of the large workloads, where the oracle cannot
solve the whole system in reasonable time.  Checked instead, with the oracle's
own code on the GPU's z:
  * the residual (s - (I + L) z)_i on sampled rows and on the hub rows,
    evaluated edge by edge in float64 (oracle.residual_rows);
  * the five quantities by their definitions (Sec. 3.2) applied to z, against
    the values the kernel reduced on the device;
  * the identities D + C = s^T z (Sec. 3.2), C_I + 2D + C = ||s||^2 and
    conservation sum z = sum s (Sec. 3.1).
"""
import numpy as np
import pytest

import oracle.fj_oracle as fo
from paper_2101_08143_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08143_gb300 import fj
    c = fj.Context(0)
    yield c
    c.close()


def _check_column(g, s, z, q, tol_rel, rng):
    n = g.n
    # residual on sampled rows + the 64 highest-degree rows
    deg = np.bincount(g.src, minlength=n) + np.bincount(g.dst, minlength=n)
    rows = np.unique(np.concatenate([rng.integers(0, n, 2000), np.argsort(-deg)[:64]]))
    sbar = s - s.mean()
    res = fo.residual_rows(n, g.src, g.dst, g.w, z, s, rows)
    scale = np.sqrt(np.sum(sbar ** 2) / n)  # rms of s_bar
    assert np.max(np.abs(res)) <= 1e-6 * scale * np.sqrt(n), np.max(np.abs(res))
    # the device-reduced quantities equal the definitions on z
    qd = fo.quantities_from_z(n, g.src, g.dst, g.w, s, z)
    for name in fo.QUANTITY_NAMES:
        assert fo.relative_error(qd[name], q[name], 1e-12 * float(s @ s)) <= tol_rel, (name, q[name], qd[name])
    # identities
    assert q["I_dc"] == pytest.approx(float(s @ z), rel=tol_rel)
    assert q["C_I"] + 2 * q["D"] + q["C"] == pytest.approx(float(s @ s), rel=tol_rel)
    assert z.sum() == pytest.approx(s.sum(), rel=1e-9)


def test_chung_lu_20m_150m(ctx):
    """n = 20,000,000, m = 150,000,000, exponent 2.1, weighted, k = 1,
    mixed precision to relative residual 1e-8."""
    import torch
    from paper_2101_08143_gb300 import fj
    spec = synth.WORKLOADS["cl_n20m_m150m_b2.1"]
    g = synth.make_graph(spec)
    s = synth.make_opinions(spec, g.n)[:, 0]
    dev = torch.device("cuda")
    with ctx.upload(g.n, torch.from_numpy(g.src).to(dev), torch.from_numpy(g.dst).to(dev),
                    torch.from_numpy(g.w).to(dev)) as dg:
        sd = torch.from_numpy(s).to(dev)
        z, q, info = ctx.solve(dg, sd, opts=fj.default_opts(tol=1e-8))
    assert info["rel_residual"] <= 1e-8
    _check_column(g, s, z.cpu().numpy(), q[0], 1e-6, np.random.default_rng(5))


def test_chung_lu_4m_40m_k256(ctx):
    """n = 4,000,000, m = 40,000,000, exponent 2.1, unit weights, k = 256
    (half uniform, half Beta(1/2, 1/2) opinions), launched as 8 x 32
    columns; 16 columns are checked."""
    import torch
    from paper_2101_08143_gb300 import fj
    spec = synth.WORKLOADS["cl_n4m_m40m_b2.1_k256"]
    g = synth.make_graph(spec)
    s = synth.make_opinions(spec, g.n)  # n x 256, column-major
    dev = torch.device("cuda")
    sd = torch.from_numpy(np.ascontiguousarray(s.T)).to(dev)  # (k, n)
    with ctx.upload(g.n, torch.from_numpy(g.src).to(dev), torch.from_numpy(g.dst).to(dev), None) as dg:
        z, q, info = ctx.solve(dg, sd, opts=fj.default_opts(tol=1e-8))
    assert info["rel_residual"] <= 1e-8
    zh = z.cpu().numpy()
    rng = np.random.default_rng(3)
    for j in list(range(0, 256, 32)) + list(range(17, 256, 32)):
        _check_column(g, s[:, j], zh[j], q[j], 1e-6, rng)
