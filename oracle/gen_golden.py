"""Write the stored expected values under tests/golden/ from the oracle alone.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Usage: python -m oracle.gen_golden [sketch | batch | paper_cd | paper_cd_dct | paper_cd_dct640]
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


# The paper's Section 6.3 sequence (three convection-diffusion problems,
# n = 500, alpha = 0, 5, 20, b = ones, 80 Arnoldi steps + 20 recycled columns,
# t = 2, at most 10 restarts, target 1e-2 relative to ||b||) with the sparse-sign
# sketch at s = 480, the largest sketch the library's handles take: exact
# recycling, the inexact variant, and the inexact variant with the stale-SAU
# rule.
PAPER_CD = dict(n=500, alpha=[0.0, 5.0, 20.0], m=80, k=20, t=2, s=480, zeta=8, rel_tol=1e-2, max_cycles=10,
                seed=231114206)


def write_paper_cd(dct=False, s=None):
    """dct: the paper's own sketch (a subsampled randomised DCT, Section 6)
    instead of the sparse sign (exact and inexact variants); s: the sketch size
    (default 480; the paper's is 8 m_max = 640)."""
    import workloads as W
    from . import sdr as O
    from .sketch import SubsampledDCT
    p = dict(PAPER_CD)
    if s is not None:
        p["s"] = s
    As = [W.make_cd_paper(p["n"], a) for a in p["alpha"]]
    N = As[0].n
    b = np.ones(N)
    S = SubsampledDCT(p["seed"], N, p["s"]) if dct else SparseSign(p["seed"], N, p["s"], p["zeta"])
    kw = dict(m=p["m"], k=p["k"], t=p["t"], rel_tol=p["rel_tol"], max_cycles=p["max_cycles"])
    doc = dict(description="Oracle runs of the paper's Section 6.3 sequence with the %s sketch at s = %d; "
                           "written by oracle.gen_golden." % ("subsampled DCT" if dct else "sparse-sign", p["s"]),
               params=p, variants={})
    variants = (("exact", True, False), ("inexact", False, False)) if dct else \
        (("exact", True, False), ("inexact", False, False), ("inexact_stale_check", False, True))
    for name, exact, stale in variants:
        t0 = time.time()
        out = O.solve_sequence(As, [b] * 3, S, exact=exact, stale_check=stale, **kw)
        runs = []
        for i, r in enumerate(out):
            steps = sum(len(c) for c in r.sres_per_cycle)
            checks = sum(len(c) for c in r.checks)
            runs.append(dict(converged=bool(r.converged), cycles=int(r.cycles), arnoldi_steps=int(steps),
                             checks=int(checks), matvecs=int(r.matvecs), sau_refreshes=int(r.sau_refreshes),
                             rel_res=float(r.res / np.linalg.norm(b)),
                             first_cycle_sres=[float(v) for v in r.sres_per_cycle[0]]))
        doc["variants"][name] = dict(problems=runs, total_matvecs=int(sum(r_["matvecs"] for r_ in runs)),
                                     oracle_seconds=time.time() - t0)
        print(name, [(r_["converged"], r_["cycles"], r_["matvecs"]) for r_ in runs], flush=True)
    name = "paper_cd_%s_s%d.json" % ("dct" if dct else "sparse_sign", p["s"])
    with open(os.path.join(GOLDEN, name), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    what = sys.argv[1:] or ["sketch"]
    if "sketch" in what:
        write_sketch_table()
    if "batch" in what:
        write_batch_large()
    if "paper_cd" in what:
        write_paper_cd()
    if "paper_cd_dct" in what:
        write_paper_cd(dct=True)
    if "paper_cd_dct640" in what:
        write_paper_cd(dct=True, s=640)
