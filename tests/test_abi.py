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
    assert lib.sdr_abi_version() == 3


def test_host_side_validation_without_gpu():
    """Invalid parameters are rejected before any CUDA call."""
    import paper_2311_14206_gb300.sdr as S
    lib = S.load_library()
    h = ctypes.c_void_p()
    bad = [S.make_params(0, 4, 2, 40, 8, 1, 1e-8), S.make_params(20, 4, 5, 40, 8, 1, 1e-8),
           S.make_params(20, 4, 2, 20, 8, 1, 1e-8), S.make_params(20, 4, 2, 800, 8, 1, 1e-8),
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
    assert ctypes.sizeof(S.sdr_stats) == 80
    assert ctypes.sizeof(S.sdr_cycle_log) == 56
    assert ctypes.sizeof(S.sdr_trace_entry) == 24
    assert len(S.KERNEL_CLASSES) == 21


def test_every_entry_point_rejects_invalid_arguments_before_cuda():
    """Each call rejects a NULL handle or an out-of-range size with INVALID_ARG
    before it touches CUDA (so this runs without a GPU)."""
    import paper_2311_14206_gb300.sdr as S
    lib = S.load_library()
    INV = 1
    i32 = ctypes.c_int32()
    dummy = ctypes.c_void_p(16)  # never dereferenced: every call below returns first
    assert lib.sdr_recycle(None, None, 0) == INV
    assert lib.sdr_sketch(None, dummy, 10, dummy) == INV
    assert lib.sdr_get_history(None, None, 0, None, None, 0, None) == INV
    assert lib.sdr_recycle_dim(None, ctypes.byref(i32)) == INV
    assert lib.sdr_recycle_export(None, 10, None, None, None) == INV
    assert lib.sdr_recycle_import(None, None, 10, 0, None, None, None) == INV
    assert lib.sdr_profile(None, 1) == INV
    assert lib.sdr_profile_get(None, None, 0, None) == INV
    assert lib.sdr_trace(None, 4) == INV
    assert lib.sdr_trace_get(None, None, 0, None) == INV
    assert lib.sdr_solve_batch(-1, None, None, None, None, None) == INV
    assert lib.sdr_solve_batch(1, None, None, None, None, None) == INV
    assert lib.sdr_recycle_batch(-1, None, None, 0) == INV
    assert lib.sdr_recycle_batch(1, None, None, 0) == INV
    # sketch without allocation: sizes outside 1 <= n < 2^31, 1 <= s <= 512,
    # 1 <= zeta <= min(s, 32), and NULL vectors
    for n, s, z, x, y in [(0, 8, 2, dummy, dummy), (1 << 31, 8, 2, dummy, dummy), (10, 0, 1, dummy, dummy),
                          (10, 513, 2, dummy, dummy), (10, 8, 0, dummy, dummy), (10, 8, 9, dummy, dummy),
                          (10, 64, 33, dummy, dummy), (10, 8, 2, None, dummy), (10, 8, 2, dummy, None)]:
        assert lib.sdr_sketch_noalloc(x, n, s, z, 1, y, None) == INV, (n, s, z)
    # adjoint helpers
    bad_csr = S.sdr_csr()
    bad_csr.n = 0
    assert lib.sdr_csr_transpose(None, dummy, dummy, dummy, dummy, None) == INV
    assert lib.sdr_csr_transpose(ctypes.byref(bad_csr), dummy, dummy, dummy, dummy, None) == INV
    assert lib.sdr_gather_values(None, dummy, 4, dummy, None) == INV
    assert lib.sdr_gather_values(dummy, dummy, -1, dummy, None) == INV
    assert lib.sdr_value_gradient(None, dummy, dummy, dummy, None) == INV
    assert lib.sdr_value_gradient(ctypes.byref(bad_csr), dummy, dummy, dummy, None) == INV
    # every status has its own text
    texts = [lib.sdr_status_string(c).decode() for c in range(8)]
    assert len(set(texts)) == 8 and "unknown status" not in texts
    assert lib.sdr_status_string(99).decode() == "unknown status"
