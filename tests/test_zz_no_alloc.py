"""The allocation-free sketch entry point against the handle-based one.

sdr_sketch_noalloc serves callers that must not let the library allocate
device memory (it works from a fixed file-scope scratch array).  Its result
must match sdr_sketch of a handle with the same parameters, call after call,
whether this file runs alone or after the rest of the suite."""
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
    seed = 231114206
    solver = P.Solver(n, m=10, k=2, t=2, s=s, zeta=zeta, seed=seed)
    rng = np.random.default_rng(n)
    xs = [torch.as_tensor(rng.standard_normal(n), device="cuda") for _ in range(2)]
    xs[1][: n // 3] = 0.0  # some all-zero tiles in the second call
    y = torch.empty(s, dtype=torch.float64, device="cuda")
    for x in xs:  # two calls in a row sharing the scratch array
        P.sdr_sketch_noalloc(x, s, zeta, seed, y)
        torch.cuda.synchronize()
        ref = P.sdr_sketch(solver.h, x, s)
        err = (y - ref).abs().max().item()
        assert err <= 1e-13 * ref.norm().item(), err
    solver.close()


def test_noalloc_rejects_out_of_range_sizes(P):
    x = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SdrError):
        P.sdr_sketch_noalloc(x, 513, 8, 1)  # s above the scratch array's 512 rows
    with pytest.raises(P.SdrError):
        P.sdr_sketch_noalloc(x, 40, 41, 1)  # zeta > s
