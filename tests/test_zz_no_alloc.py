"""The allocation-free sketch entry point against the handle-based one and
the oracle.

sdr_sketch_noalloc serves callers that must not let the library allocate
device memory: code that runs while another component owns the device's
memory (a framework's pool, a budget fixed at start-up), and paths where a
cudaMalloc, which may synchronise the device, cannot be taken.  It works from
a fixed file-scope scratch array.  Its result must equal sdr_sketch of a
handle with the same parameters bit for bit (the handle's n_max equals n
here), call after call, whether this file runs alone or after the rest of
the suite, and match the oracle's SparseSign within rounding."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2311_14206_gb300 as P
    return P


@pytest.mark.parametrize("n,s,zeta", [(5000, 120, 8), (300000, 480, 8), (777, 37, 3)])
def test_noalloc_matches_handle_sketch_two_calls(P, n, s, zeta):
    from oracle.sketch import SparseSign
    seed = 231114206
    solver = P.Solver(n, m=10, k=2, t=2, s=s, zeta=zeta, seed=seed)
    S = SparseSign(seed, n, s, zeta)
    rng = np.random.default_rng(n)
    xs = [rng.standard_normal(n) for _ in range(2)]
    xs[1][: n // 3] = 0.0  # some all-zero tiles in the second call
    y = torch.empty(s, dtype=torch.float64, device="cuda")
    for xh in xs:  # two calls in a row sharing the scratch array
        x = torch.as_tensor(xh, device="cuda")
        P.sdr_sketch_noalloc(x, s, zeta, seed, y)
        torch.cuda.synchronize()
        ref = P.sdr_sketch(solver.h, x, s)
        assert torch.equal(y, ref), (y - ref).abs().max().item()
        yo = S.apply(xh)
        err = np.abs(y.cpu().numpy() - yo).max()
        assert err <= 1e-13 * np.linalg.norm(yo), err
    solver.close()


def test_noalloc_zero_and_nonfinite_inputs(P):
    s, zeta, seed, n = 64, 4, 7, 3000
    y = torch.full((s,), 5.0, dtype=torch.float64, device="cuda")
    P.sdr_sketch_noalloc(torch.zeros(n, dtype=torch.float64, device="cuda"), s, zeta, seed, y)
    torch.cuda.synchronize()
    assert torch.equal(y, torch.zeros_like(y))  # x == 0 gives y == 0
    for bad in (math.nan, math.inf, -math.inf):
        x = torch.ones(n, dtype=torch.float64, device="cuda")
        x[1234] = bad
        P.sdr_sketch_noalloc(x, s, zeta, seed, y)
        torch.cuda.synchronize()
        assert torch.isnan(y).all(), bad  # a non-finite x is reported as NaN, never as a finite y
    # and the scratch array serves the next finite call correctly
    x = torch.arange(n, dtype=torch.float64, device="cuda")
    P.sdr_sketch_noalloc(x, s, zeta, seed, y)
    torch.cuda.synchronize()
    from oracle.sketch import SparseSign
    yo = SparseSign(seed, n, s, zeta).apply(x.cpu().numpy())
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-13 * np.linalg.norm(yo)


def test_noalloc_rejects_out_of_range_sizes(P):
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SdrError):
        P.sdr_sketch_noalloc(x, 513, 8, 1)  # s above the scratch array's 512 rows
    with pytest.raises(P.SdrError):
        P.sdr_sketch_noalloc(x, 40, 41, 1)  # zeta > s
    with pytest.raises(P.SdrError):  # y too short for s: rejected before the C call
        P.sdr_sketch_noalloc(x, 40, 4, 1, torch.empty(39, dtype=torch.float64, device="cuda"))
    with pytest.raises(P.SdrError):  # x of the wrong type
        P.sdr_sketch_noalloc(x.float(), 40, 4, 1)
