"""Write the stored expected values under tests/golden/ from the oracle alone.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Usage: python -m oracle.gen_golden
"""
import json
import os

import numpy as np

from .sketch import sketch_indices

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


if __name__ == "__main__":
    write_sketch_table()
