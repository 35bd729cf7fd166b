"""The C-ABI library builds, loads, and exports every symbol of include/fj.h.
No compute call is made here (this file runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2101_08143_gb300 import fj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fj_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_symbols_exported():
    lib = fj.load()
    names = _declared_symbols()
    assert "fj_solve" in names and "fj_graph_upload" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_header_constants_match_the_binding():
    text = open(os.path.join(ROOT, "include", "fj.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (FJ_[A-Z_]+) (\d+)u", text)}
    assert defs["FJ_HOST_PTRS"] == fj.FJ_HOST_PTRS
    assert defs["FJ_DEVICE_PTRS"] == fj.FJ_DEVICE_PTRS
    assert defs["FJ_MERGE_DUPLICATES"] == fj.FJ_MERGE_DUPLICATES
    assert defs["FJ_TWO_SOLVES"] == fj.FJ_TWO_SOLVES


def test_version_and_defaults():
    assert "sm_103a" in fj.version()
    o = fj.default_opts()
    assert o.tol == 1e-10 and o.precision == fj.PREC_MIXED and o.max_iter > 0


def test_null_arguments_are_rejected_without_a_device():
    lib = fj.load()
    assert lib.fj_solve_ex(None, None, 1, None, None, None, None, None) == fj.FJ_ERR_ARG
    assert b"non-NULL" in lib.fj_last_error()
    assert lib.fj_graph_stats(None, None, None, None) == fj.FJ_ERR_ARG
    assert lib.fj_set_max_blocks(None, 3) == fj.FJ_ERR_ARG
    assert lib.fj_destroy(None) == fj.FJ_OK


def test_built_for_sm_103a():
    from paper_2101_08143_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_serving_arguments_rejected_without_a_device():
    import ctypes as C
    lib = fj.load()
    t = C.c_uint64()
    assert lib.fj_submit(None, None, 1, None, None, C.byref(t)) == fj.FJ_ERR_ARG
    assert lib.fj_poll(None, 1, 0, None, None) == fj.FJ_ERR_ARG
    assert lib.fj_serve_config(None, 1, 0, 0) == fj.FJ_ERR_ARG


def test_new_entry_points_reject_null_arguments_without_a_device():
    import ctypes as C
    lib = fj.load()
    out = C.c_void_p()
    assert lib.fj_graph_lcc(None, None, C.byref(out)) == fj.FJ_ERR_ARG
    assert b"non-NULL" in lib.fj_last_error()
    assert lib.fj_graph_node_ids(None, None, None) == fj.FJ_ERR_ARG
    info = fj.Info()
    assert lib.fj_solve_warm(None, None, 1, None, None, None, None, None, C.byref(info)) == fj.FJ_ERR_ARG
    assert b"z0" in lib.fj_last_error()


def test_tune_layout_and_null_arguments_without_a_device():
    import ctypes as C
    text = open(os.path.join(ROOT, "include", "fj.h")).read()
    assert int(re.search(r"#define FJ_TUNE_MAX (\d+)", text).group(1)) == fj.FJ_TUNE_MAX
    # int32 best, int32 count, int32[16] blocks, then double[16] ms at offset 72
    assert C.sizeof(fj.TuneResult) == 72 + 8 * fj.FJ_TUNE_MAX
    assert fj.TuneResult.ms.offset == 72
    lib = fj.load()
    res = fj.TuneResult()
    assert lib.fj_tune(None, None, 1, None, None, 3, C.byref(res)) == fj.FJ_ERR_ARG
    assert b"non-NULL" in lib.fj_last_error()
    assert lib.fj_tune(None, None, 1, None, None, 0, C.byref(res)) == fj.FJ_ERR_ARG


def test_info_layout_and_set_grid_arguments_without_a_device():
    import ctypes as C
    # int32 x2, double x2, int32 status, columns, blocks, uint32 warnings,
    # double t_begin_ms, t_end_ms, int32 batched, reserved
    assert fj.Info.blocks.offset == 32 and fj.Info.warnings.offset == 36
    assert fj.Info.t_begin_ms.offset == 40 and fj.Info.batched.offset == 56 and C.sizeof(fj.Info) == 64
    text = open(os.path.join(ROOT, "include", "fj.h")).read()
    assert int(re.search(r"#define FJ_WARN_OPINION_RANGE (\d+)u", text).group(1)) == fj.FJ_WARN_OPINION_RANGE
    lib = fj.load()
    assert lib.fj_set_grid(None, 4) == fj.FJ_ERR_ARG
    assert b"fj_set_grid" in lib.fj_last_error()


def test_binding_declares_every_header_function():
    """The ctypes binding gives a prototype to every function of fj.h."""
    text = open(os.path.join(ROOT, "include", "fj.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(fj_[a-z0-9_]+)\s*\(", text))
    assert names and not (names - set(fj._SIGNATURES)), sorted(names - set(fj._SIGNATURES))
