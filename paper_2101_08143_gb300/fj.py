"""Python binding of libfj (include/fj.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts numpy arrays / torch CUDA tensors into pointers and sizes.  Importing
it loads libfj.so and raises if the library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FJ_OK = 0
FJ_PENDING = 1
FJ_ERR_ARG = -1
FJ_ERR_GRAPH = -2
FJ_ERR_OOM = -3
FJ_ERR_ADMIT = -4
FJ_ERR_NOT_CONVERGED = -5
FJ_ERR_NUMERIC = -6
FJ_ERR_TIMEOUT = -7
FJ_ERR_CUDA = -8
FJ_ERR_TICKET = -9

FJ_HOST_PTRS = 0
FJ_DEVICE_PTRS = 1
FJ_MERGE_DUPLICATES = 2
FJ_TWO_SOLVES = 4
FJ_QUANTITY_TOL = 8
FJ_WARN_OPINION_RANGE = 1

PREC_MIXED = 0
PREC_FP64 = 1
PREC_FP32 = 2

QUANTITY_NAMES = ("C_I", "D", "P", "C", "I_dc")
FJ_TUNE_MAX = 16


class FJError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fj error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("precision", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("device_ms", ctypes.c_double),
                ("status", ctypes.c_int32), ("columns", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("warnings", ctypes.c_uint32),
                ("t_begin_ms", ctypes.c_double), ("t_end_ms", ctypes.c_double),
                ("batched", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Quant(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in QUANTITY_NAMES]


class Layout(ctypes.Structure):
    _fields_ = [("chunk_len", ctypes.c_int32), ("sell_max", ctypes.c_int32)]


FJ_LAYOUT_TUNE_MAX = 16


class LayoutTuneResult(ctypes.Structure):
    _fields_ = [("best", Layout), ("count", ctypes.c_int32), ("tried", Layout * FJ_LAYOUT_TUNE_MAX),
                ("ms", ctypes.c_double * FJ_LAYOUT_TUNE_MAX)]


class TuneResult(ctypes.Structure):
    _fields_ = [("best", ctypes.c_int32), ("count", ctypes.c_int32),
                ("blocks", ctypes.c_int32 * FJ_TUNE_MAX), ("ms", ctypes.c_double * FJ_TUNE_MAX)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "fj_default_opts": (None, [ctypes.POINTER(Opts)]),
    "fj_last_error": (ctypes.c_char_p, []),
    "fj_version": (ctypes.c_char_p, []),
    "fj_kernel_launches": (ctypes.c_int64, []),
    "fj_create": (ctypes.c_int32, [ctypes.c_int, ctypes.POINTER(_P)]),
    "fj_destroy": (ctypes.c_int32, [_P]),
    "fj_set_stream": (ctypes.c_int32, [_P, _P]),
    "fj_set_max_blocks": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "fj_set_grid": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "fj_graph_upload": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P,
                                         ctypes.c_uint32, ctypes.POINTER(_P)]),
    "fj_graph_free": (ctypes.c_int32, [_P, _P]),
    "fj_graph_stats": (ctypes.c_int32, [_P, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "fj_solve_ex": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P, _P,
                                     ctypes.POINTER(Opts), ctypes.POINTER(Info)]),
    "fj_graph_lcc": (ctypes.c_int32, [_P, _P, ctypes.POINTER(_P)]),
    "fj_graph_node_ids": (ctypes.c_int32, [_P, _P, _P]),
    "fj_solve_warm": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P, _P, _P,
                                       ctypes.POINTER(Opts), ctypes.POINTER(Info)]),
    "fj_solve": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P,
                                  ctypes.POINTER(Opts), ctypes.POINTER(Info)]),
    "fj_quantities": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P,
                                       ctypes.POINTER(Opts), ctypes.POINTER(Info)]),
    "fj_serve_config": (ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32]),
    "fj_submit": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, ctypes.POINTER(Opts),
                                   ctypes.POINTER(ctypes.c_uint64)]),
    "fj_submit_edges": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P,
                                         ctypes.c_int32, _P, ctypes.POINTER(Opts),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "fj_poll": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.c_int32, _P, ctypes.POINTER(Info)]),
    "fj_tune": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, ctypes.POINTER(Opts), ctypes.c_int32,
                                 ctypes.POINTER(TuneResult)]),
    "fj_solve_fixed": (ctypes.c_int32, [_P, _P, ctypes.c_int32, _P, _P, _P, ctypes.POINTER(Opts),
                                        ctypes.POINTER(Info)]),
    "fj_debug_barrier": (ctypes.c_int32, [ctypes.c_int64, ctypes.c_int32]),
    "fj_graph_update_weights": (ctypes.c_int32, [_P, _P, ctypes.c_int64, _P, _P, _P, ctypes.c_uint32]),
    "fj_set_layout": (ctypes.c_int32, [_P, ctypes.POINTER(Layout)]),
    "fj_graph_layout": (ctypes.c_int32, [_P, ctypes.POINTER(Layout)]),
    "fj_tune_layout": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, ctypes.c_uint32,
                                        ctypes.c_int32, _P, ctypes.POINTER(Opts), ctypes.c_int32,
                                        ctypes.POINTER(LayoutTuneResult)]),
    "fj_serve_pack": (ctypes.c_int32, [_P, ctypes.c_int64]),
    "fj_solve_batch": (ctypes.c_int32, [_P, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.POINTER(Opts),
                                        _P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libfj.so (building it first if needed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise FJError(FJ_ERR_CUDA, f"libfj.so not found at {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code, what=""):
    if code != FJ_OK:
        msg = load().fj_last_error().decode()
        raise FJError(code, f"{what}: {msg}" if what else msg)


def default_opts(**kw) -> Opts:
    o = Opts()
    load().fj_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _is_torch_cuda(x):
    return hasattr(x, "is_cuda") and x.is_cuda


class Graph:
    def __init__(self, ctx: "Context", handle):
        self.ctx = ctx
        self.handle = handle

    def stats(self):
        n = ctypes.c_int64()
        nnz = ctypes.c_int64()
        wt = ctypes.c_int32()
        _check(load().fj_graph_stats(self.handle, ctypes.byref(n), ctypes.byref(nnz),
                                     ctypes.byref(wt)), "fj_graph_stats")
        return {"n": n.value, "nnz": nnz.value, "weighted": bool(wt.value)}

    def lcc(self) -> "Graph":
        """The subgraph induced on the largest connected component."""
        h = _P()
        _check(load().fj_graph_lcc(self.ctx.handle, self.handle, ctypes.byref(h)), "fj_graph_lcc")
        return Graph(self.ctx, h)

    def node_ids(self) -> np.ndarray:
        """Node i's id in the parent graph (i for an uploaded graph)."""
        ids = np.empty(self.stats()["n"], dtype=np.int32)
        _check(load().fj_graph_node_ids(self.ctx.handle, self.handle, _P(ids.ctypes.data)),
               "fj_graph_node_ids")
        return ids

    def layout(self):
        lay = Layout()
        _check(load().fj_graph_layout(self.handle, ctypes.byref(lay)), "fj_graph_layout")
        return {"chunk_len": lay.chunk_len, "sell_max": lay.sell_max}

    def update_weights(self, src, dst, w):
        """fj_graph_update_weights: new weights for existing pairs (host
        numpy arrays, or torch CUDA tensors: int32, int32, float32)."""
        lib = load()
        if _is_torch_cuda(src):
            count = int(src.numel())
            rc = lib.fj_graph_update_weights(self.ctx.handle, self.handle, count, _P(src.data_ptr()),
                                             _P(dst.data_ptr()), _P(w.data_ptr()), FJ_DEVICE_PTRS)
        else:
            src = np.ascontiguousarray(src, dtype=np.int32)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            w = np.ascontiguousarray(w, dtype=np.float32)
            rc = lib.fj_graph_update_weights(self.ctx.handle, self.handle, int(src.shape[0]),
                                             _P(src.ctypes.data), _P(dst.ctypes.data), _P(w.ctypes.data),
                                             FJ_HOST_PTRS)
        _check(rc, "fj_graph_update_weights")

    def free(self):
        if self.handle:
            _check(load().fj_graph_free(self.ctx.handle, self.handle), "fj_graph_free")
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


class Context:
    """A libfj context on one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load()
        h = _P()
        _check(lib.fj_create(device, ctypes.byref(h)), "fj_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load().fj_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream_ptr: int | None):
        _check(load().fj_set_stream(self.handle, _P(stream_ptr or 0)), "fj_set_stream")

    def set_max_blocks(self, nblocks: int):
        _check(load().fj_set_max_blocks(self.handle, int(nblocks)), "fj_set_max_blocks")

    def set_grid(self, nblocks: int):
        """fj_set_grid: later solves run on exactly nblocks blocks (0: default)."""
        _check(load().fj_set_grid(self.handle, int(nblocks)), "fj_set_grid")

    # ------------------------------------------------------------- graphs
    def upload(self, n, src, dst, w=None, merge_duplicates=False) -> Graph:
        """Edge list -> device CSR.  numpy arrays (host) or torch CUDA tensors
        (device); w=None means unit weights.  A pair listed twice raises
        FjError unless merge_duplicates, which adds the repeats' weights."""
        h = _P()
        if _is_torch_cuda(src):
            m = int(src.numel())
            args = (src.data_ptr(), dst.data_ptr(), w.data_ptr() if w is not None else None)
            flags = FJ_DEVICE_PTRS
            keep = None
        else:
            src = np.ascontiguousarray(src, dtype=np.int32)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
            m = int(src.shape[0])
            keep = (src, dst, w)
            args = (src.ctypes.data, dst.ctypes.data, None if w is None else w.ctypes.data)
            flags = FJ_HOST_PTRS
        if merge_duplicates:
            flags |= FJ_MERGE_DUPLICATES
        rc = load().fj_graph_upload(self.handle, int(n), m, _P(args[0]), _P(args[1]),
                                    _P(args[2]), flags, ctypes.byref(h))
        del keep
        _check(rc, "fj_graph_upload")
        return Graph(self, h)

    def set_layout(self, chunk_len=None, sell_max=None):
        """Layout of later uploads (None, None: the defaults)."""
        if chunk_len is None and sell_max is None:
            _check(load().fj_set_layout(self.handle, None), "fj_set_layout")
            return
        lay = Layout(512 if chunk_len is None else chunk_len, 64 if sell_max is None else sell_max)
        _check(load().fj_set_layout(self.handle, ctypes.byref(lay)), "fj_set_layout")

    def tune_layout(self, n, src, dst, w, s, opts: Opts | None = None, repeats: int = 3,
                    merge_duplicates=False):
        """fj_tune_layout on host or device (torch) edge arrays and opinions;
        returns {"best": (chunk_len, sell_max), "ms": {(chunk_len, sell_max): ms}}."""
        lib = load()
        o = Opts()
        lib.fj_default_opts(ctypes.byref(o))
        if opts is not None:
            o = Opts(opts.tol, opts.inner_tol, opts.precision, opts.max_iter, opts.max_refine, opts.flags)
        keep = []
        if _is_torch_cuda(src):
            flags = FJ_DEVICE_PTRS
            m = int(src.numel())
            sp, dp = src.data_ptr(), dst.data_ptr()
            wp = w.data_ptr() if w is not None else None
        else:
            flags = FJ_HOST_PTRS
            src = np.ascontiguousarray(src, dtype=np.int32)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
            keep += [src, dst, w]
            m = int(src.shape[0])
            sp, dp = src.ctypes.data, dst.ctypes.data
            wp = w.ctypes.data if w is not None else None
        if merge_duplicates:
            flags |= FJ_MERGE_DUPLICATES
        if _is_torch_cuda(s):
            k = 1 if s.dim() == 1 else int(s.shape[0])
            o.flags = (o.flags & ~FJ_DEVICE_PTRS) | FJ_DEVICE_PTRS
            s_ptr = s.data_ptr()
        else:
            s2 = np.asfortranarray(np.asarray(s, dtype=np.float64).reshape(n, -1))
            keep.append(s2)
            k = s2.shape[1]
            o.flags = o.flags & ~FJ_DEVICE_PTRS
            s_ptr = s2.ctypes.data
        res = LayoutTuneResult()
        _check(lib.fj_tune_layout(self.handle, int(n), m, _P(sp), _P(dp), _P(wp), flags, k, _P(s_ptr),
                                  ctypes.byref(o), int(repeats), ctypes.byref(res)), "fj_tune_layout")
        del keep
        return {"best": (res.best.chunk_len, res.best.sell_max),
                "ms": {(res.tried[i].chunk_len, res.tried[i].sell_max): res.ms[i] for i in range(res.count)}}

    def upload_edges(self, edges, merge_duplicates=False) -> Graph:
        """Upload a synth.EdgeList."""
        return self.upload(edges.n, edges.src, edges.dst, edges.w, merge_duplicates)

    # -------------------------------------------------------------- solve
    def solve(self, graph: Graph, s, want_z=True, want_quant=True, opts: Opts | None = None,
              z_out=None, raise_on_error=True, z0=None):
        """Solve (I + L) z = s for the columns of s.

        s: numpy float64 (n,) or (n, k) [host], or a torch float64 CUDA tensor
        of shape (k, n) / (n,) whose rows are the columns (column-major n x k
        memory) [device].  Returns (z, quantities, info); z is a numpy (n, k)
        array for host input, or the z_out / new torch tensor for device input.
        z0: optional initial guess in the same form as s (fj_solve_warm).
        """
        lib = load()
        o = Opts() if opts is None else opts
        if opts is None:
            lib.fj_default_opts(ctypes.byref(o))
        else:
            o = Opts(opts.tol, opts.inner_tol, opts.precision, opts.max_iter,
                     opts.max_refine, opts.flags)
        n = graph.stats()["n"]
        if _is_torch_cuda(s):
            import torch
            k = 1 if s.dim() == 1 else int(s.shape[0])
            if not s.is_contiguous() or s.dtype != torch.float64 or s.numel() != n * k:
                raise ValueError("device s must be contiguous float64 with n*k elements")
            z = None
            if want_z:
                z = z_out if z_out is not None else torch.empty_like(s)
            sp, zp = s.data_ptr(), (z.data_ptr() if z is not None else None)
            if z0 is not None and (not z0.is_contiguous() or z0.dtype != torch.float64
                                   or z0.numel() != n * k):
                raise ValueError("device z0 must be contiguous float64 shaped like s")
            z0p = z0.data_ptr() if z0 is not None else None
            o.flags = (o.flags & ~FJ_DEVICE_PTRS) | FJ_DEVICE_PTRS
            keep = None
        else:
            s = np.asarray(s, dtype=np.float64)
            squeeze = s.ndim == 1
            s2 = s.reshape(n, -1)
            k = s2.shape[1]
            sf = np.asfortranarray(s2)
            z = None
            if want_z:
                if z_out is not None:
                    z = z_out
                    if z.dtype != np.float64 or not z.flags.f_contiguous or z.size != n * k:
                        raise ValueError("host z_out must be F-contiguous float64 with n*k elements")
                else:
                    z = np.empty((n, k), dtype=np.float64, order="F")
            sp = sf.ctypes.data
            zp = z.ctypes.data if z is not None else None
            o.flags = (o.flags & ~FJ_DEVICE_PTRS) | FJ_HOST_PTRS
            z0f = None if z0 is None else np.asfortranarray(
                np.asarray(z0, dtype=np.float64).reshape(n, k))
            z0p = z0f.ctypes.data if z0f is not None else None
            keep = (sf, z0f)
        quant = (Quant * k)() if want_quant else None
        info = Info()
        qp = ctypes.cast(quant, _P) if quant is not None else None
        if z0 is None:
            rc = lib.fj_solve_ex(self.handle, graph.handle, k, _P(sp), _P(zp), qp,
                                 ctypes.byref(o), ctypes.byref(info))
        else:
            rc = lib.fj_solve_warm(self.handle, graph.handle, k, _P(sp), _P(z0p), _P(zp), qp,
                                   ctypes.byref(o), ctypes.byref(info))
        del keep
        if raise_on_error:
            _check(rc, "fj_solve_ex" if z0 is None else "fj_solve_warm")
        qs = None
        if quant is not None:
            qs = [{name: getattr(quant[j], name) for name in QUANTITY_NAMES} for j in range(k)]
        if z is not None and not _is_torch_cuda(s) and squeeze and z.ndim == 2:
            z = z[:, 0]
        d = info.as_dict()
        d["rc"] = rc
        return z, qs, d

    def solve_batch(self, graphs, s_list, want_z=True, opts: Opts | None = None, raise_on_error=True):
        """fj_solve_batch: many problems in packed launches.

        graphs: list of Graph; s_list: per problem a host numpy float64 (n,)
        or (n, k) array, or (all of them) torch float64 CUDA tensors of shape
        (k, n) / (n,).  Returns (rc, [(z, quantities, info) per problem])."""
        lib = load()
        o = Opts()
        lib.fj_default_opts(ctypes.byref(o))
        if opts is not None:
            o = Opts(opts.tol, opts.inner_tol, opts.precision, opts.max_iter, opts.max_refine, opts.flags)
        count = len(graphs)
        device = _is_torch_cuda(s_list[0])
        ks, sp, zp, zs, keep = [], [], [], [], []
        for g, sv in zip(graphs, s_list):
            n = g.stats()["n"]
            if device:
                k = 1 if sv.dim() == 1 else int(sv.shape[0])
                if not sv.is_contiguous() or sv.numel() != n * k:
                    raise ValueError("device s must be contiguous float64 with n*k elements")
                z = None
                if want_z:
                    import torch
                    z = torch.empty_like(sv)
                sp.append(sv.data_ptr())
                zp.append(z.data_ptr() if z is not None else None)
            else:
                s2 = np.asfortranarray(np.asarray(sv, dtype=np.float64).reshape(n, -1))
                k = s2.shape[1]
                z = np.empty((n, k), dtype=np.float64, order="F") if want_z else None
                keep.append(s2)
                sp.append(s2.ctypes.data)
                zp.append(z.ctypes.data if z is not None else None)
            ks.append(k)
            zs.append(z)
        o.flags = (o.flags & ~FJ_DEVICE_PTRS) | (FJ_DEVICE_PTRS if device else FJ_HOST_PTRS)
        quants = [(Quant * k)() for k in ks]
        infos = (Info * count)()
        ga = (_P * count)(*[g.handle for g in graphs])
        ka = (ctypes.c_int32 * count)(*ks)
        sa = (_P * count)(*sp)
        za = (_P * count)(*zp) if want_z else None
        qa = (_P * count)(*[ctypes.cast(q, _P) for q in quants])
        rc = lib.fj_solve_batch(self.handle, count, ga, ka, sa, za, qa, ctypes.byref(o), infos)
        del keep
        if raise_on_error and rc != FJ_OK:
            _check(rc, "fj_solve_batch")
        out = []
        for i in range(count):
            qs = [{name: getattr(quants[i][j], name) for name in QUANTITY_NAMES} for j in range(ks[i])]
            d = infos[i].as_dict()
            out.append((zs[i], qs, d))
        return rc, out

    def quantities(self, graph: Graph, s, opts: Opts | None = None):
        _, q, info = self.solve(graph, s, want_z=False, want_quant=True, opts=opts)
        return q, info

    def tune(self, graph: Graph, s, opts: Opts | None = None, repeats: int = 3):
        """fj_tune: time the solve of s on graph under each candidate grid and
        keep the fastest for later solves of as many columns in the same
        precision class.  s as for solve().  Returns {"best": blocks (0 =
        default sizing), "grids": [(blocks, median ms), ...]}."""
        lib = load()
        o = Opts()
        lib.fj_default_opts(ctypes.byref(o))
        if opts is not None:
            o = Opts(opts.tol, opts.inner_tol, opts.precision, opts.max_iter,
                     opts.max_refine, opts.flags)
        n = graph.stats()["n"]
        if _is_torch_cuda(s):
            import torch
            k = 1 if s.dim() == 1 else int(s.shape[0])
            if not s.is_contiguous() or s.dtype != torch.float64 or s.numel() != n * k:
                raise ValueError("device s must be contiguous float64 with n*k elements")
            keep, sp = s, s.data_ptr()
            o.flags = (o.flags & ~FJ_DEVICE_PTRS) | FJ_DEVICE_PTRS
        else:
            sf = np.asfortranarray(np.asarray(s, dtype=np.float64).reshape(n, -1))
            k = sf.shape[1]
            keep, sp = sf, sf.ctypes.data
            o.flags = (o.flags & ~FJ_DEVICE_PTRS) | FJ_HOST_PTRS
        res = TuneResult()
        rc = lib.fj_tune(self.handle, graph.handle, k, _P(sp), ctypes.byref(o), int(repeats),
                         ctypes.byref(res))
        del keep
        _check(rc, "fj_tune")
        return {"best": res.best,
                "grids": [(res.blocks[i], res.ms[i]) for i in range(res.count)]}


class Ticket:
    """A submitted request: its id and the number of opinion vectors."""

    def __init__(self, tid: int, k: int):
        self.id = tid
        self.k = k


def _host_s(s, n):
    s = np.asarray(s, dtype=np.float64)
    s2 = np.asfortranarray(s.reshape(n, -1))
    return s2, s2.shape[1]


def _serve_opts(opts):
    o = Opts()
    load().fj_default_opts(ctypes.byref(o))
    if opts is not None:
        o = Opts(opts.tol, opts.inner_tol, opts.precision, opts.max_iter, opts.max_refine,
                 opts.flags & ~FJ_DEVICE_PTRS)
    return o


def serve_config(ctx: "Context", max_inflight=0, mem_budget_bytes=0, max_blocks_per_request=-1):
    _check(load().fj_serve_config(ctx.handle, int(max_inflight), int(mem_budget_bytes),
                                  int(max_blocks_per_request)), "fj_serve_config")


def serve_pack(ctx: "Context", max_nodes: int):
    """Requests with at most max_nodes nodes are solved in packed batches
    (0: none)."""
    _check(load().fj_serve_pack(ctx.handle, int(max_nodes)), "fj_serve_pack")


def submit(ctx: "Context", graph: "Graph", s, opts: Opts | None = None) -> Ticket:
    """Queue a solve on a resident graph; s is host float64 (n,) or (n, k)."""
    n = graph.stats()["n"]
    s2, k = _host_s(s, n)
    t = ctypes.c_uint64()
    o = _serve_opts(opts)
    _check(load().fj_submit(ctx.handle, graph.handle, k, _P(s2.ctypes.data), ctypes.byref(o),
                            ctypes.byref(t)), "fj_submit")
    return Ticket(t.value, k)


def submit_edges(ctx: "Context", n, src, dst, w, s, opts: Opts | None = None,
                 merge_duplicates=False) -> Ticket:
    """Queue a request that carries its own edge list (host arrays); a pair
    listed twice fails the request unless merge_duplicates."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    s2, k = _host_s(s, n)
    t = ctypes.c_uint64()
    o = _serve_opts(opts)
    if merge_duplicates:
        o.flags |= FJ_MERGE_DUPLICATES
    _check(load().fj_submit_edges(ctx.handle, int(n), int(src.shape[0]), _P(src.ctypes.data),
                                  _P(dst.ctypes.data), _P(None if w is None else w.ctypes.data), k,
                                  _P(s2.ctypes.data), ctypes.byref(o), ctypes.byref(t)),
           "fj_submit_edges")
    return Ticket(t.value, k)


def poll(ctx: "Context", ticket: Ticket, timeout_us: int = -1):
    """Returns (rc, quantities or None, info dict).  rc == FJ_PENDING while
    the request runs."""
    quant = (Quant * ticket.k)()
    info = Info()
    rc = load().fj_poll(ctx.handle, ticket.id, int(timeout_us), ctypes.cast(quant, _P),
                        ctypes.byref(info))
    if rc == FJ_PENDING:
        return rc, None, None
    qs = [{name: getattr(quant[j], name) for name in QUANTITY_NAMES} for j in range(ticket.k)]
    d = info.as_dict()
    d["rc"] = rc
    return rc, qs, d


def version() -> str:
    return load().fj_version().decode()
