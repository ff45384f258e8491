"""Write the stored expected values under tests/golden/ from the oracle alone.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Usage: python -m oracle.gen_golden [sketch | batch]
"""
import json
import os
import sys
import time

import numpy as np

from .sketch import SparseSign, sketch_indices

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(os.path.dirname(HERE), "tests", "golden")

SKETCH_CASES = [
    dict(seed=0, s=120, zeta=8, ncols=64),
    dict(seed=231114206, s=120, zeta=8, ncols=64),
    dict(seed=231114206, s=480, zeta=8, ncols=64),
    dict(seed=231114206, s=100, zeta=8, ncols=64),
    dict(seed=231114206, s=300, zeta=8, ncols=64),
    dict(seed=231114206, s=400, zeta=8, ncols=64),
    dict(seed=12345, s=37, zeta=3, ncols=64),
]


def write_sketch_table():
    cases = []
    for c in SKETCH_CASES:
        rows, signs = sketch_indices(c["seed"], c["s"], c["zeta"], np.arange(c["ncols"]))
        cases.append(dict(c, rows=rows.tolist(), signs=signs.tolist()))
    doc = dict(
        description="Rows and signs of the first columns of the hash-defined sparse-sign "
                    "embedding (SplitMix64 words, Floyd sampling); written by oracle.gen_golden.",
        cases=cases)
    os.makedirs(GOLDEN, exist_ok=True)
    with open(os.path.join(GOLDEN, "sketch_indices.json"), "w") as f:
        json.dump(doc, f, separators=(",", ":"))


# The batched workload (64 2D convection-diffusion systems, sides U{32..512},
# 5-system sequences, m = 40, k = 10, t = 2, s = 100, zeta = 8, tol 1e-8): two
# of its largest systems, one whose sequence converges throughout (51) and one
# whose fifth solve stalls at this sketch size (59), solved by the oracle.
BATCH_CASES = (51, 59)
BATCH_PARAMS = dict(m=40, k=10, t=2, s=100, zeta=8, rel_tol=1e-8, max_cycles=200, seq=5, eps=1e-3,
                    seed=231114206, count=64, nmin=32, nmax=512, samples=64)


def batch_system(i, p=BATCH_PARAMS):
    """Matrices and right-hand sides of system i of the batched workload."""
    import workloads as W
    n, conv = W.batch_systems(p["count"], p["nmin"], p["nmax"])[i]
    A0 = W.make_cd2d(n, conv)
    dvec = W.diag_perturbation(A0.n, tag=i)
    As = list(W.sequence_matrices(A0, p["seq"], p["eps"], dvec))
    bs = [W.rhs(A0.n, 1000 * i + j) for j in range(p["seq"])]
    return n, conv, As, bs


def write_batch_large():
    from . import sdr as O
    p = BATCH_PARAMS
    doc = dict(description="Oracle solves of two large systems of the batched workload (exact recycling "
                           "along each 5-system sequence); written by oracle.gen_golden.",
               params=p, systems=[])
    for i in BATCH_CASES:
        n, conv, As, bs = batch_system(i)
        S = SparseSign(p["seed"], As[0].n, p["s"], p["zeta"])
        t0 = time.time()
        out = O.solve_sequence(As, bs, S, m=p["m"], k=p["k"], t=p["t"], rel_tol=p["rel_tol"],
                               max_cycles=p["max_cycles"])
        idx = np.sort(np.random.default_rng([7, i]).choice(As[0].n, p["samples"], replace=False))
        solves = []
        for j, r in enumerate(out):
            solves.append(dict(converged=bool(r.converged), cycles=int(r.cycles), matvecs=int(r.matvecs),
                               rel_res=float(r.res / np.linalg.norm(bs[j])), xnorm=float(np.linalg.norm(r.x)),
                               x_samples=r.x[idx].tolist(), first_cycle_sres=[float(v) for v in r.sres_per_cycle[0]]))
        doc["systems"].append(dict(index=i, side=n, conv=list(conv), N=int(As[0].n), sample_index=idx.tolist(),
                                   solves=solves, oracle_seconds=time.time() - t0))
        print(i, n, [(s_["converged"], s_["cycles"], f"{s_['rel_res']:.2e}") for s_ in solves], flush=True)
    with open(os.path.join(GOLDEN, "batch64_large_systems.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    what = sys.argv[1:] or ["sketch"]
    if "sketch" in what:
        write_sketch_table()
    if "batch" in what:
        write_batch_large()
