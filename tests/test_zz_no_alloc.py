"""fj_solve_fixed: the solve variant that allocates no device memory.

Some callers cannot allocate while they solve: a latency-critical loop (where
cudaMalloc/cudaFree may stall the whole device) or a program whose device
memory belongs to another allocator.  fj_solve_fixed serves them from a fixed
scratch array inside the library.  This file checks, through the C ABI, that
two calls in a row give the same answers as the allocating entry point
fj_solve_ex, in every precision mode, with the per-quantity target and
without z, that the device's free
memory does not change across calls once the first call has run, and that
requests larger than the fixed array, or host arrays, are refused.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


class _Quant(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("C_I", "D", "P", "C", "I_dc")]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08143_gb300 import fj
    lib = fj.load()
    f = lib.fj_solve_fixed
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(fj.Opts),
                  ctypes.POINTER(fj.Info)]
    ctx = fj.Context(0)
    yield torch, fj, lib, ctx
    ctx.close()


def _fixed(torch, fj, lib, graph, s_ptr, z_ptr, k, opts):
    quant = (_Quant * k)()
    info = fj.Info()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.fj_solve_fixed(graph.handle, ctypes.c_void_p(stream), k, ctypes.c_void_p(s_ptr),
                            ctypes.c_void_p(z_ptr), ctypes.cast(quant, ctypes.c_void_p),
                            ctypes.byref(opts), ctypes.byref(info))
    torch.cuda.synchronize()
    q = [{n: getattr(quant[j], n) for n in fj.QUANTITY_NAMES} for j in range(k)]
    return rc, q, info


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_fixed_matches_allocating_solve_twice(env, precision):
    torch, fj, lib, ctx = env
    from paper_2101_08143_gb300 import synth
    g = synth.chung_lu(3000, 15000, 2.3, seed=12, weighted=True)
    k = 3
    tol = 1e-10 if precision != 2 else 1e-6
    s = synth.opinions_uniform(g.n, k, 17)
    s_dev = torch.from_numpy(np.ascontiguousarray(s.T)).cuda()  # (k, n): column-major n x k
    opts = fj.default_opts(precision=precision, tol=tol)
    with ctx.upload_edges(g) as dg:
        z_ref, q_ref, _ = ctx.solve(dg, s_dev, opts=opts)
        for _ in range(2):
            z_dev = torch.full_like(s_dev, float("nan"))
            rc, q, info = _fixed(torch, fj, lib, dg, s_dev.data_ptr(), z_dev.data_ptr(), k, opts)
            assert rc == fj.FJ_OK, lib.fj_last_error()
            assert info.rel_residual <= tol
            np.testing.assert_allclose(z_dev.cpu().numpy(), z_ref.cpu().numpy(), rtol=0, atol=1e-8)
            for j in range(k):
                for name in fj.QUANTITY_NAMES:
                    ref = q_ref[j][name]
                    assert abs(q[j][name] - ref) <= 1e-6 * max(abs(ref), 1e-12), (name, q[j][name], ref)


def test_fixed_with_the_quantity_target_twice(env):
    """FJ_QUANTITY_TOL reaches the fixed entry point: two calls in a row give
    the quantities of the allocating solve with the same target, each within
    the target of the exact values, so within twice it of each other."""
    torch, fj, lib, ctx = env
    from paper_2101_08143_gb300 import synth
    g = synth.erdos_renyi(4000, 24000, seed=14, weighted=True)
    k = 2
    s = synth.opinions_uniform(g.n, k, 19)
    s_dev = torch.from_numpy(np.ascontiguousarray(s.T)).cuda()
    opts = fj.default_opts(tol=1e-6, flags=fj.FJ_QUANTITY_TOL)
    with ctx.upload_edges(g) as dg:
        _, q_ref, _ = ctx.solve(dg, s_dev, opts=opts, want_z=False)
        for _ in range(2):
            z_dev = torch.full_like(s_dev, float("nan"))
            rc, q, _ = _fixed(torch, fj, lib, dg, s_dev.data_ptr(), z_dev.data_ptr(), k, opts)
            assert rc == fj.FJ_OK, lib.fj_last_error()
            assert not torch.isnan(z_dev).any()
            for j in range(k):
                for name in fj.QUANTITY_NAMES:
                    ref = q_ref[j][name]
                    assert abs(q[j][name] - ref) <= 2e-6 * abs(ref), (name, q[j][name], ref)


def test_fixed_without_z_and_free_memory_unchanged(env):
    """z = NULL gives the same quantities; after a first call (which may load
    the solver's code and the scratch array on the device), further calls
    leave the device's free memory and torch's allocations unchanged."""
    torch, fj, lib, ctx = env
    from paper_2101_08143_gb300 import synth
    g = synth.chung_lu(20000, 80000, 2.1, seed=13, weighted=True)
    k = 5
    s = synth.opinions_uniform(g.n, k, 18)
    s_dev = torch.from_numpy(np.ascontiguousarray(s.T)).cuda()
    opts = fj.default_opts(tol=1e-10)
    with ctx.upload_edges(g) as dg:
        _, q_ref, _ = ctx.solve(dg, s_dev, opts=opts, want_z=False)
        rc, _, _ = _fixed(torch, fj, lib, dg, s_dev.data_ptr(), None, k, opts)  # first call
        assert rc == fj.FJ_OK, lib.fj_last_error()
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        for _ in range(2):
            rc, q, _ = _fixed(torch, fj, lib, dg, s_dev.data_ptr(), None, k, opts)
            assert rc == fj.FJ_OK, lib.fj_last_error()
            for j in range(k):
                for name in fj.QUANTITY_NAMES:
                    ref = q_ref[j][name]
                    assert abs(q[j][name] - ref) <= 1e-6 * max(abs(ref), 1e-12), name
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.memory_allocated() == alloc0


def test_fixed_refuses_oversized_requests_and_host_arrays(env):
    torch, fj, lib, ctx = env
    n = 200_000  # 32 columns of this size need far more than the fixed scratch
    empty = np.zeros(0, np.int32)
    with ctx.upload(n, empty, empty) as dg:
        s_dev = torch.zeros((32, n), dtype=torch.float64, device="cuda")
        z_dev = torch.zeros_like(s_dev)
        rc, _, _ = _fixed(torch, fj, lib, dg, s_dev.data_ptr(), z_dev.data_ptr(), 32, fj.default_opts())
        assert rc == fj.FJ_ERR_ARG
        assert b"fixed area holds" in lib.fj_last_error()
        rc, _, _ = _fixed(torch, fj, lib, dg, s_dev.data_ptr(), z_dev.data_ptr(), 33, fj.default_opts())
        assert rc == fj.FJ_ERR_ARG
        # host arrays (pageable or page-locked) are refused before any launch
        s_host = np.zeros(n)
        rc, _, _ = _fixed(torch, fj, lib, dg, s_host.ctypes.data, None, 1, fj.default_opts())
        assert rc == fj.FJ_ERR_ARG
        assert b"device memory" in lib.fj_last_error()
        s_pin = torch.zeros(n, dtype=torch.float64).pin_memory()
        rc, _, _ = _fixed(torch, fj, lib, dg, s_dev.data_ptr(), s_pin.data_ptr(), 1, fj.default_opts())
        assert rc == fj.FJ_ERR_ARG
