"""The C-ABI library builds, loads and exports every entry point of include/sdr.h
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sdr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdr_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("sdr_create", "sdr_solve", "sdr_recycle", "sdr_destroy"):
        assert f in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_2311_14206_gb300 import _build
    lib = ctypes.CDLL(_build.LIB)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing
    assert lib.sdr_abi_version() == 2


def test_host_side_validation_without_gpu():
    """Invalid parameters are rejected before any CUDA call."""
    import paper_2311_14206_gb300.sdr as S
    lib = S.load_library()
    h = ctypes.c_void_p()
    bad = [S.make_params(0, 4, 2, 40, 8, 1, 1e-8), S.make_params(20, 4, 5, 40, 8, 1, 1e-8),
           S.make_params(20, 4, 2, 20, 8, 1, 1e-8), S.make_params(20, 4, 2, 600, 8, 1, 1e-8),
           S.make_params(20, 4, 2, 40, 0, 1, 1e-8), S.make_params(20, 40, 2, 100, 8, 1, 1e-8),
           S.make_params(20, 4, 2, 40, 8, 1, -1.0),
           S.make_params(20, 4, 2, 40, 8, 1, 1e-8, precision=7),
           S.make_params(20, 4, 2, 40, 8, 1, 1e-8, precision=S.SDR_PREC_F32_REFINED, inner_rel_tol=2.0)]
    for p in bad:
        assert lib.sdr_create(ctypes.byref(p), 1000, None, ctypes.byref(h)) == 1
    assert lib.sdr_solve(None, None, None, None, None) == 1
    assert lib.sdr_destroy(None) == 0


def test_struct_layouts_match_the_header():
    """The binding's structs have the header's sizes (natural alignment)."""
    import paper_2311_14206_gb300.sdr as S
    assert ctypes.sizeof(S.sdr_params) == 88
    assert ctypes.sizeof(S.sdr_csr) == 48
    assert ctypes.sizeof(S.sdr_stats) == 72
    assert ctypes.sizeof(S.sdr_cycle_log) == 56
    assert ctypes.sizeof(S.sdr_trace_entry) == 24
    assert len(S.KERNEL_CLASSES) == 21
