"""The binding checks every array before its raw pointer reaches the library
(no GPU needed: each case is rejected on the host, before any CUDA call).

The library reads or writes exactly n (or nnz, or s) elements behind each
pointer, so an array of the wrong size, type or layout would become an
out-of-bounds device access; the binding turns it into a Python error."""
import pytest

torch = pytest.importorskip("torch")

import paper_2311_14206_gb300.sdr as S  # noqa: E402
from paper_2311_14206_gb300.adjoint import AdjointPair  # noqa: E402


def csr(n=4, nnz=6, rp=None):
    rowptr = torch.zeros(n + 1 if rp is None else rp, dtype=torch.int32)
    return S.CSRDevice(n, rowptr, torch.zeros(nnz, dtype=torch.int32), torch.zeros(nnz, dtype=torch.float64))


def vec(n, dtype=torch.float64):
    return torch.zeros(n, dtype=dtype)


def test_csr_sizes_then_placement():
    with pytest.raises(ValueError):
        csr(rp=4).c_struct()  # rowptr needs n + 1 entries
    A = csr()
    A.col = torch.zeros(5, dtype=torch.int32)
    with pytest.raises(ValueError):
        A.c_struct()  # col and val differ in length
    A = csr()
    A.val32 = torch.zeros(5, dtype=torch.float32)
    with pytest.raises(ValueError):
        A.c_struct()
    with pytest.raises(TypeError):
        csr().c_struct()  # right sizes, but host memory
    with pytest.raises(ValueError):
        S.CSRDevice(0, vec(1, torch.int32), vec(0, torch.int32), vec(0)).c_struct()


def test_solve_vectors():
    S.load_library()
    A = csr()
    with pytest.raises(ValueError):
        S.sdr_solve(None, A, vec(3), vec(4))  # b shorter than n
    with pytest.raises(ValueError):
        S.sdr_solve(None, A, vec(4), vec(5))  # x longer than n
    with pytest.raises(TypeError):
        S.sdr_solve(None, A, vec(4, torch.float32), vec(4))
    with pytest.raises(TypeError):
        S.sdr_solve(None, A, vec(4), torch.zeros(8, dtype=torch.float64)[::2])  # not contiguous
    with pytest.raises(TypeError):
        S.sdr_solve(None, A, vec(4), vec(4))  # host memory


def test_batch_lengths_and_vectors():
    A = csr()
    with pytest.raises(ValueError):
        S.sdr_solve_batch([None, None], [A], [vec(4)], [vec(4)])
    with pytest.raises(ValueError):
        S.sdr_solve_batch([None], [A], [vec(4)], [vec(2)])
    with pytest.raises(ValueError):
        S.sdr_recycle_batch([None, None], [A])


def test_sketch_size_checked_against_the_handle():
    fake = 0x5D12  # never passed to the library: every call below stops first
    S._HANDLE_S[fake] = 40
    try:
        with pytest.raises(ValueError):
            S.sdr_sketch(fake, vec(10), 41)
        with pytest.raises(ValueError):
            S.sdr_recycle_export(fake, 10, 39)
        U = torch.zeros(10, 2, dtype=torch.float64)
        with pytest.raises(ValueError):
            S.sdr_recycle_import(fake, None, U, torch.zeros(39, 2, dtype=torch.float64))  # s rows
        with pytest.raises(ValueError):
            S.sdr_recycle_import(fake, None, U, torch.zeros(40, 3, dtype=torch.float64))  # k columns
        with pytest.raises(ValueError):
            S.sdr_recycle_import(fake, None, torch.zeros(10, dtype=torch.float64))  # U not 2-D
        with pytest.raises(TypeError):
            S.sdr_recycle_import(fake, None, U)  # host memory
    finally:
        S._HANDLE_S.pop(fake, None)
    with pytest.raises(TypeError):
        S.sdr_sketch(None, vec(10, torch.float32), 40)


def test_adjoint_pattern_checked():
    with pytest.raises(ValueError):
        AdjointPair(4, vec(4, torch.int32), vec(6, torch.int32), 10, 2, 2, 20)  # rowptr needs n + 1 entries
    with pytest.raises(TypeError):
        AdjointPair(4, vec(5, torch.int64), vec(6, torch.int32), 10, 2, 2, 20)
