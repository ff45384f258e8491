"""The batched form at the workload's own sizes: two of the largest systems of
the 64-system batched workload (2D convection-diffusion, sides 509 and 495,
5-system sequences with exact recycling, m = 40, k = 10, s = 100), solved in
lockstep by sdr_solve_batch, against the oracle's solves of the same
sequences (tests/golden/batch64_large_systems.json, written by
oracle/gen_golden.py from the oracle alone).

System 51 converges in every solve.  In system 59 the second solve stalls in
the oracle (sketch size s = 100 for up to 51 columns is too small an embedding
for that recycled space; the true residual stops following the sketched one).
Such a stall is decided by rounding over some two hundred restarts on a weak
embedding: the GPU either stalls there too, at a true residual within a factor
of ten of the oracle's, or converges, its true residual then checked against
tol.  Once the two sides part there (one stalled, one converged), their recycle
spaces differ, and the later solves of that system are checked for a true
residual below tol only.

Cycle counts: these solves run 40 to 55 cycles on a weak embedding, and the
GPU's and the oracle's rounding steer them apart over that many restarts (each
cycle's recycle space agrees with the oracle's to about 1e-6 in angle, the
bar of the cycle-replay test, and the differences compound); the bar is 20 %
of the oracle's count (at least one cycle), while the solution, the true
residual and the first cycle's sketched residuals keep the strict bars."""
import json
import os

import numpy as np
import pytest

from oracle import sdr as osdr
from oracle.gen_golden import batch_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch64_large_systems.json")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2311_14206_gb300 as P
    return P


def test_batch64_large_systems_match_oracle(P):
    gold = json.load(open(GOLDEN))
    p = gold["params"]
    systems = []
    for sysg in gold["systems"]:
        n, conv, As, bs = batch_system(sysg["index"])
        assert As[0].n == sysg["N"]
        systems.append((sysg, As, bs))
    handles = [P.Solver(As[0].n, p["m"], p["k"], p["t"], p["s"], p["zeta"], p["seed"], p["rel_tol"],
                        max_cycles=p["max_cycles"], stream=torch.cuda.Stream()) for _, As, _ in systems]
    hs = [h.h for h in handles]
    parted = [False] * len(systems)
    for j in range(p["seq"]):
        A_j = [P.CSRDevice.from_numpy(As[j]) for _, As, _ in systems]
        b_j = [torch.as_tensor(bs[j], device="cuda") for _, _, bs in systems]
        xs = [torch.zeros_like(b) for b in b_j]
        if j > 0:
            P.sdr_recycle_batch(hs, A_j, 0)
        st, stats = P.sdr_solve_batch(hs, A_j, b_j, xs)
        for si, ((sysg, As, bs), x, s_, h) in enumerate(zip(systems, xs, stats, handles)):
            ref = sysg["solves"][j]
            xh = x.cpu().numpy()
            bn = np.linalg.norm(bs[j])
            rel = np.linalg.norm(bs[j] - osdr.csr_matvec(As[j], xh)) / bn
            where = f"system {sysg['index']} solve {j}: gpu cycles {s_['cycles']} res {s_['final_rel_res']:.2e}, " \
                    f"oracle cycles {ref['cycles']} res {ref['rel_res']:.2e}"
            if parted[si]:  # the recycle spaces differ since an earlier stall on one side only
                if s_["converged"]:
                    assert rel < p["rel_tol"] * (1 + 1e-9), where
                continue
            if not ref["converged"] and s_["converged"]:  # the stall did not recur under the GPU's rounding
                assert rel < p["rel_tol"] * (1 + 1e-9), where
                parted[si] = True
                continue
            assert bool(s_["converged"]) == ref["converged"], where
            if ref["converged"]:
                assert rel < p["rel_tol"] * (1 + 1e-9), where
                assert abs(s_["cycles"] - ref["cycles"]) <= max(1, 0.2 * ref["cycles"]), \
                    (where, s_["cycles"], ref["cycles"])
                xo = np.asarray(ref["x_samples"])
                assert abs(np.linalg.norm(xh) - ref["xnorm"]) <= 1e-6 * ref["xnorm"], where
                assert np.max(np.abs(xh[sysg["sample_index"]] - xo)) <= 1e-6 * ref["xnorm"], where
            else:
                # both sides stall at the cycle cap, far above the tolerance
                assert s_["cycles"] == p["max_cycles"] and rel > 100 * p["rel_tol"], (where, rel)
                assert 0.1 < rel / ref["rel_res"] < 10.0, (where, rel, ref["rel_res"])
            if j == 0:  # the first cycle of a fresh solve: per-step sres at the parity bar
                sres, _ = P.sdr_get_history(h.h)
                r = np.asarray(ref["first_cycle_sres"])
                g = np.asarray(sres[:r.size])
                assert np.all(np.abs(g - r) <= 1e-8 * r + 1e-13 * bn), where
    for h in handles:
        h.close()
