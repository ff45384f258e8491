"""Python binding of libsdr.so (include/sdr.h): argument marshalling only.

The functions carry the C names (sdr_create, sdr_solve, sdr_recycle,
sdr_destroy, ...).  Device arrays are torch CUDA tensors; their data pointers
and the current torch stream are handed to the library, which does all the
work in its own kernels.  There is no fallback: if the library is missing or
no GPU is present the calls raise.
"""
import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

LIB_PATH = _build.LIB

SDR_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory", 4: "not converged",
          5: "breakdown", 6: "rank", 7: "not implemented"}


class sdr_params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("k", ctypes.c_int32), ("t", ctypes.c_int32), ("s", ctypes.c_int32),
                ("zeta", ctypes.c_int32), ("seed", ctypes.c_uint64), ("rel_tol", ctypes.c_double),
                ("safety0", ctypes.c_double), ("max_cycles", ctypes.c_int32), ("persist_safety", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("test_flags", ctypes.c_int32), ("inner_rel_tol", ctypes.c_double),
                ("stale_check", ctypes.c_int32), ("sketch_kind", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


SDR_PREC_F64 = 0
SDR_PREC_F32_REFINED = 1


class sdr_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("val32", ctypes.c_void_p)]


class sdr_stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int32), ("converged", ctypes.c_int32), ("matvecs", ctypes.c_int32),
                ("sketches", ctypes.c_int32), ("true_res_evals", ctypes.c_int32), ("arnoldi_steps", ctypes.c_int32),
                ("recycle_dim", ctypes.c_int32), ("full_svd_cycles", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("sau_refreshes", ctypes.c_int32), ("refresh_matvecs", ctypes.c_int32), ("final_res", ctypes.c_double),
                ("tol", ctypes.c_double), ("final_rel_res", ctypes.c_double), ("bnorm", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


KERNEL_CLASSES = ["solve_init", "residual0", "cycle_init", "spmv_dots", "update_sketch", "step_dense",
                  "check_gemv", "check_residual", "ce_formC", "recycle_gemm", "recycle_sau", "sketch",
                  "ce_rinv", "ce_M", "ce_svd", "ce_eig", "ce_invit", "ce_select", "ce_finish", "ce_sketches",
                  "refine"]


class sdr_kernel_time(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32), ("pad", ctypes.c_int32), ("total_ms", ctypes.c_double)]


class sdr_trace_entry(ctypes.Structure):
    _fields_ = [("cls", ctypes.c_int32), ("stream", ctypes.c_int32), ("start_us", ctypes.c_double),
                ("end_us", ctypes.c_double)]


class sdr_cycle_log(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("checks", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("ell", ctypes.c_int32), ("kprime", ctypes.c_int32), ("kh", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("svd_sweeps", ctypes.c_int32), ("res", ctypes.c_double),
                ("sres", ctypes.c_double), ("safety", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libsdr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2311_14206_gb300._build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "sdr_create": ([P(sdr_params), i64, vp, P(vp)], i32),
        "sdr_solve": ([vp, P(sdr_csr), vp, vp, P(sdr_stats)], i32),
        "sdr_recycle": ([vp, P(sdr_csr), i32], i32),
        "sdr_destroy": ([vp], i32),
        "sdr_sketch": ([vp, vp, i64, vp], i32),
        "sdr_sketch_noalloc": ([vp, i64, i32, i32, ctypes.c_uint64, vp, vp], i32),
        "sdr_get_history": ([vp, P(ctypes.c_double), i32, P(i32), P(sdr_cycle_log), i32, P(i32)], i32),
        "sdr_recycle_dim": ([vp, P(i32)], i32),
        "sdr_get_givens": ([vp, P(ctypes.c_double), P(ctypes.c_double), i32, P(i32)], i32),
        "sdr_set_sketch_draws": ([vp, i64, vp, vp], i32),
        "sdr_recycle_export": ([vp, i64, vp, vp, vp], i32),
        "sdr_recycle_import": ([vp, P(sdr_csr), i64, i32, vp, vp, vp], i32),
        "sdr_profile": ([vp, i32], i32),
        "sdr_profile_get": ([vp, P(sdr_kernel_time), i32, P(i32)], i32),
        "sdr_trace": ([vp, i32], i32),
        "sdr_trace_get": ([vp, P(sdr_trace_entry), i32, P(i32)], i32),
        "sdr_csr_transpose": ([P(sdr_csr), vp, vp, vp, vp, vp], i32),
        "sdr_solve_batch": ([i32, P(vp), P(sdr_csr), P(vp), P(vp), P(sdr_stats)], i32),
        "sdr_recycle_batch": ([i32, P(vp), P(sdr_csr), i32], i32),
        "sdr_gather_values": ([vp, vp, i64, vp, vp], i32),
        "sdr_value_gradient": ([P(sdr_csr), vp, vp, vp, vp], i32),
        "sdr_status_string": ([i32], ctypes.c_char_p),
        "sdr_abi_version": ([], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


class SdrError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


def _check(st, where, ok=(SDR_OK,)):
    if st not in ok:
        raise SdrError(st, where)
    return st


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_len(t, n, name):
    """t is a tensor of n elements (ValueError otherwise).  The wrappers check
    the sizes of all their arrays first, then their type and placement."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, the library uses {n}")


def _device_array(t, n, name, dtype=torch.float64, device=None):
    """Check t before its raw pointer reaches the library, which reads or writes
    exactly n elements of dtype there: a tensor of n elements, contiguous, of
    dtype, on a CUDA device (the given one, if any).  Raises ValueError or
    TypeError."""
    _check_len(t, n, name)
    if t.dtype != dtype or not t.is_contiguous() or not t.is_cuda:
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if device is not None and t.device != device:
        raise TypeError(f"{name} is on {t.device}, the other arrays on {device}")
    return t


# The sketch size s of each handle created through this module: the library
# writes s-element sketches into buffers the caller passes, and the ABI has no
# call that reports s.
_HANDLE_S = {}


def _handle_s(h):
    return _HANDLE_S.get(h.value if isinstance(h, ctypes.c_void_p) else h)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class CSRDevice:
    """Square CSR matrix held in torch CUDA tensors (int32 / int32 / float64,
    plus an optional float32 copy of the values for the refined form)."""

    n: int
    rowptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor
    val32: torch.Tensor = None

    @classmethod
    def from_numpy(cls, A, device="cuda", with_f32=False):
        val = torch.as_tensor(A.val, dtype=torch.float64).to(device)
        return cls(A.n, torch.as_tensor(A.rowptr, dtype=torch.int32).to(device),
                   torch.as_tensor(A.col, dtype=torch.int32).to(device), val,
                   val.to(torch.float32) if with_f32 else None)

    def c_struct(self) -> sdr_csr:
        if not self.n >= 1:
            raise ValueError(f"CSR order n = {self.n}")
        nnz = int(self.val.numel())
        _check_len(self.rowptr, self.n + 1, "rowptr")
        _check_len(self.col, nnz, "col")
        if self.val32 is not None:
            _check_len(self.val32, nnz, "val32")
        _device_array(self.rowptr, self.n + 1, "rowptr", torch.int32)
        dev = self.rowptr.device
        _device_array(self.col, nnz, "col", torch.int32, dev)
        _device_array(self.val, nnz, "val", torch.float64, dev)
        v32 = 0
        if self.val32 is not None:
            v32 = _device_array(self.val32, nnz, "val32", torch.float32, dev).data_ptr()
        return sdr_csr(self.n, int(self.val.numel()), self.rowptr.data_ptr(), self.col.data_ptr(),
                       self.val.data_ptr(), v32)


def make_params(m, k, t, s, zeta, seed, rel_tol, safety0=1.4, max_cycles=200, persist_safety=0,
                force_svd=False, precision=SDR_PREC_F64, inner_rel_tol=0.0, graphs=True,
                stale_check=False, integer_recycle=False, sketch_kind=0) -> sdr_params:
    p = sdr_params(m, k, t, s, zeta, seed, rel_tol, safety0, max_cycles, persist_safety)
    p.precision = precision
    p.test_flags = (1 if force_svd else 0) | (0 if graphs else 2) | (4 if integer_recycle else 0)
    p.inner_rel_tol = inner_rel_tol
    p.stale_check = 1 if stale_check else 0
    p.sketch_kind = sketch_kind
    return p


def sdr_create(params: sdr_params, n_max: int, stream=None) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    st = lib.sdr_create(ctypes.byref(params), n_max, stream if stream is not None else _stream(), ctypes.byref(h))
    _check(st, "sdr_create")
    _HANDLE_S[h.value] = int(params.s)
    return h


def sdr_solve(h, A: CSRDevice, b: torch.Tensor, x: torch.Tensor, allow_not_converged=True, allow=()):
    """Solve in place into x; returns (status, stats dict).  Statuses other than
    OK (and NOT_CONVERGED when allow_not_converged) raise SdrError, unless
    listed in `allow` (for instance SDR_ERR_BREAKDOWN = 5)."""
    lib = load_library()
    _check_len(b, A.n, "b")
    _check_len(x, A.n, "x")
    _device_array(b, A.n, "b")
    _device_array(x, A.n, "x", device=b.device)
    csr = A.c_struct()
    if A.val.device != b.device:
        raise TypeError(f"A is on {A.val.device}, b and x on {b.device}")
    stats = sdr_stats()
    st = lib.sdr_solve(h, ctypes.byref(csr), _ptr(b), _ptr(x), ctypes.byref(stats))
    _check(st, "sdr_solve", ok=((0, 4) if allow_not_converged else (0,)) + tuple(allow))
    return st, stats.as_dict()


def sdr_solve_batch(handles, As, bs, xs, allow_not_converged=True):
    """Solve len(handles) independent systems in lockstep (one handle, stream and
    recycle space each); x arrays are overwritten.  Returns (status, [stats])."""
    lib = load_library()
    cnt = len(handles)
    if not (len(As) == len(bs) == len(xs) == cnt):
        raise ValueError(f"{cnt} handles, {len(As)} matrices, {len(bs)} right-hand sides, {len(xs)} solutions")
    for A, b, x in zip(As, bs, xs):
        _check_len(b, A.n, "b")
        _check_len(x, A.n, "x")
    for A, b, x in zip(As, bs, xs):
        _device_array(b, A.n, "b")
        _device_array(x, A.n, "x", device=b.device)
    H = (ctypes.c_void_p * cnt)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    C = (sdr_csr * cnt)(*[A.c_struct() for A in As])
    B = (ctypes.c_void_p * cnt)(*[b.data_ptr() for b in bs])
    X = (ctypes.c_void_p * cnt)(*[x.data_ptr() for x in xs])
    S = (sdr_stats * cnt)()
    st = lib.sdr_solve_batch(cnt, H, C, B, X, S)
    _check(st, "sdr_solve_batch", ok=(0, 4) if allow_not_converged else (0,))
    return st, [S[i].as_dict() for i in range(cnt)]


def sdr_recycle_batch(handles, As, mode=0):
    lib = load_library()
    cnt = len(handles)
    if As is not None and len(As) != cnt:
        raise ValueError(f"{cnt} handles, {len(As)} matrices")
    H = (ctypes.c_void_p * cnt)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    C = (sdr_csr * cnt)(*[A.c_struct() for A in As]) if As is not None else None
    return _check(lib.sdr_recycle_batch(cnt, H, C, mode), "sdr_recycle_batch")


def sdr_recycle(h, A_next: CSRDevice = None, mode: int = 0):
    lib = load_library()
    csr = A_next.c_struct() if A_next is not None else None
    return _check(lib.sdr_recycle(h, ctypes.byref(csr) if csr is not None else None, mode), "sdr_recycle")


def sdr_destroy(h):
    _HANDLE_S.pop(h.value if isinstance(h, ctypes.c_void_p) else h, None)
    return load_library().sdr_destroy(h)


def _check_s(h, s, where):
    hs = _handle_s(h)
    if hs is not None and s != hs:
        raise ValueError(f"{where}: s = {s}, but the handle sketches to {hs} rows")


def sdr_sketch(h, x: torch.Tensor, s: int) -> torch.Tensor:
    _check_s(h, s, "sdr_sketch")
    _device_array(x, x.numel(), "x")
    y = torch.empty(s, dtype=torch.float64, device=x.device)
    _check(load_library().sdr_sketch(h, _ptr(x), x.numel(), _ptr(y)), "sdr_sketch")
    return y


def sdr_sketch_noalloc(x: torch.Tensor, s: int, zeta: int, seed: int, y: torch.Tensor = None) -> torch.Tensor:
    """y = S x through the allocation-free entry point (y preallocated by the
    caller, or here by torch when y is None).  x and y must be contiguous
    float64 CUDA tensors on one device, y with at least s entries: the C call
    takes raw pointers and would read or write past a smaller array."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
        raise SdrError(1, "sdr_sketch_noalloc: x must be a contiguous float64 CUDA tensor")
    if y is None:
        y = torch.empty(s, dtype=torch.float64, device=x.device)
    if not y.is_cuda or y.dtype != torch.float64 or not y.is_contiguous() or y.device != x.device:
        raise SdrError(1, "sdr_sketch_noalloc: y must be a contiguous float64 CUDA tensor on x's device")
    if y.numel() < s:
        raise SdrError(1, f"sdr_sketch_noalloc: y has {y.numel()} entries, fewer than s = {s}")
    with torch.cuda.device(x.device):
        _check(load_library().sdr_sketch_noalloc(_ptr(x), x.numel(), s, zeta, seed, _ptr(y), _stream()),
               "sdr_sketch_noalloc")
    return y


def sdr_get_history(h, cap_steps=1 << 15, cap_cycles=512):
    lib = load_library()
    sres = (ctypes.c_double * cap_steps)()
    logs = (sdr_cycle_log * cap_cycles)()
    ns, nc = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.sdr_get_history(h, sres, cap_steps, ctypes.byref(ns), logs, cap_cycles, ctypes.byref(nc)),
           "sdr_get_history")
    log = [{f: getattr(logs[i], f) for f, _ in sdr_cycle_log._fields_} for i in range(min(nc.value, cap_cycles))]
    return list(sres[:min(ns.value, cap_steps)]), log


def sdr_set_sketch_draws(h, signs, rows):
    """Random draws of a DCT-sketch handle: signs (n values +-1) and rows (s
    strictly increasing frequencies), host arrays."""
    import numpy as np
    sg = np.ascontiguousarray(np.asarray(signs), dtype=np.int8)
    rw = np.ascontiguousarray(np.asarray(rows), dtype=np.int32)
    _check(load_library().sdr_set_sketch_draws(h, sg.size, sg.ctypes.data_as(ctypes.c_void_p),
                                               rw.ctypes.data_as(ctypes.c_void_p)), "sdr_set_sketch_draws")


def sdr_get_givens(h, cap_steps=1 << 15):
    """(sines, cosines) of the Givens rotations of every Arnoldi step of the last solve."""
    s = (ctypes.c_double * cap_steps)()
    c = (ctypes.c_double * cap_steps)()
    n = ctypes.c_int32()
    _check(load_library().sdr_get_givens(h, s, c, cap_steps, ctypes.byref(n)), "sdr_get_givens")
    k = min(n.value, cap_steps)
    return list(s[:k]), list(c[:k])


def sdr_recycle_dim(h) -> int:
    k = ctypes.c_int32()
    _check(load_library().sdr_recycle_dim(h, ctypes.byref(k)), "sdr_recycle_dim")
    return k.value


def sdr_recycle_export(h, n: int, s: int, device="cuda"):
    _check_s(h, s, "sdr_recycle_export")
    kd = sdr_recycle_dim(h)
    U = torch.empty((kd, n), dtype=torch.float64, device=device)  # row c = column c (column-major n x kd)
    SU = torch.empty((kd, s), dtype=torch.float64, device=device)
    SAU = torch.empty((kd, s), dtype=torch.float64, device=device)
    if kd:
        _check(load_library().sdr_recycle_export(h, n, _ptr(U), _ptr(SU), _ptr(SAU)), "sdr_recycle_export")
    return U.T, SU.T, SAU.T


def sdr_recycle_import(h, A: CSRDevice, U: torch.Tensor, SU: torch.Tensor = None, SAU: torch.Tensor = None):
    """U, SU, SAU given as (n x k), (s x k), (s x k) arrays; stored column-major."""
    if U.dim() != 2:
        raise ValueError("U must be an n x k array")
    n, kd = U.shape
    hs = _handle_s(h)
    for name, X in (("SU", SU), ("SAU", SAU)):
        if X is not None and (X.dim() != 2 or X.shape[1] != kd or (hs is not None and X.shape[0] != hs)):
            raise ValueError(f"{name} has shape {tuple(X.shape)}, expected (s, {kd})"
                             + (f" with s = {hs}" if hs is not None else ""))
    Uc = _device_array(U.T.contiguous(), n * kd, "U")
    SUc = _device_array(SU.T.contiguous(), SU.numel(), "SU", device=Uc.device) if SU is not None else None
    SAUc = _device_array(SAU.T.contiguous(), SAU.numel(), "SAU", device=Uc.device) if SAU is not None else None
    csr = A.c_struct() if A is not None else None
    st = load_library().sdr_recycle_import(h, ctypes.byref(csr) if csr is not None else None, n, kd, _ptr(Uc),
                                           _ptr(SUc), _ptr(SAUc))
    return _check(st, "sdr_recycle_import")


def sdr_profile(h, enable=True):
    return _check(load_library().sdr_profile(h, 1 if enable else 0), "sdr_profile")


def sdr_profile_get(h):
    """{class name: (launches, total ms)} of the library's kernels since sdr_profile."""
    arr = (sdr_kernel_time * len(KERNEL_CLASSES))()
    n = ctypes.c_int32()
    _check(load_library().sdr_profile_get(h, arr, len(KERNEL_CLASSES), ctypes.byref(n)), "sdr_profile_get")
    return {KERNEL_CLASSES[i]: (arr[i].launches, arr[i].total_ms) for i in range(min(n.value, len(KERNEL_CLASSES)))}


def sdr_trace(h, cap):
    return _check(load_library().sdr_trace(h, int(cap)), "sdr_trace")


def sdr_trace_get(h):
    """[(class name, stream, start us, end us)] of the traced launches."""
    n = ctypes.c_int32()
    lib = load_library()
    _check(lib.sdr_trace_get(h, None, 0, ctypes.byref(n)), "sdr_trace_get")
    arr = (sdr_trace_entry * max(n.value, 1))()
    _check(lib.sdr_trace_get(h, arr, n.value, ctypes.byref(n)), "sdr_trace_get")
    return [(KERNEL_CLASSES[e.cls], e.stream, e.start_us, e.end_us) for e in arr[:n.value]]


class Solver:
    """Convenience wrapper owning one handle (GMRES-SDR for one system size)."""

    def __init__(self, n_max, m, k, t, s, zeta=8, seed=231114206, rel_tol=1e-8, safety0=1.4, max_cycles=200,
                 persist_safety=0, force_svd=False, precision=SDR_PREC_F64, inner_rel_tol=0.0, graphs=True,
                 stream=None, stale_check=False, integer_recycle=False, sketch_kind=0):
        self.params = make_params(m, k, t, s, zeta, seed, rel_tol, safety0, max_cycles, persist_safety, force_svd,
                                  precision, inner_rel_tol, graphs, stale_check, integer_recycle, sketch_kind)
        self.n_max, self.s = n_max, s
        self.stream = stream  # a torch.cuda.Stream the handle issues on (None: the current stream)
        self.h = sdr_create(self.params, n_max,
                            ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)

    def solve(self, A: CSRDevice, b: torch.Tensor, x: torch.Tensor = None):
        if x is None:
            x = torch.zeros_like(b)
        st, stats = sdr_solve(self.h, A, b, x)
        return x, st, stats

    def recycle(self, A_next=None, mode=0):
        return sdr_recycle(self.h, A_next, mode)

    def set_sketch_draws(self, signs, rows):
        """DCT-sketch handles: the random signs (n of them) and the s selected rows."""
        if len(rows) != self.s:
            raise SdrError(1, f"set_sketch_draws: {len(rows)} rows for s = {self.s}")
        sdr_set_sketch_draws(self.h, signs, rows)

    def history(self):
        return sdr_get_history(self.h)

    def close(self):
        if self.h is not None:
            sdr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
