"""Plant plausible mistakes in copies of the oracle and check that a pin fails.

Each mutation edits the source of the oracle module in memory (on the CPU),
loads the edited copy as a separate module and runs the pins against it.  A
mutation that no pin notices would mean the pins leave that part unchecked."""
import importlib.util
import inspect
import sys
import types

import numpy as np
import pytest

import oracle_pins as P
from oracle import sdr, sketch

SDR_MUTATIONS = [
    ("SAV drops the h(j+1,j) term", "SV[:, :j + 2] @ H[:j + 2, j]", "SV[:, :j + 1] @ H[:j + 1, j]"),
    ("MGS update with the wrong sign", "w = w - V[:, i] * H[i, j]", "w = w + V[:, i] * H[i, j]"),
    ("back substitution with R transposed", "back_substitute(R, Q.T @ Sr0)", "back_substitute(R.T, Q.T @ Sr0)"),
    ("sketched residual with a sign error", "np.linalg.norm(Sr0 - SAW @ y)", "np.linalg.norm(Sr0 + SAW @ y)"),
    ("smallest instead of largest |mu|", "np.lexsort((idx, -mu.real, -np.abs(mu)))",
     "np.lexsort((idx, -mu.real, np.abs(mu)))"),
    ("M_ell transposed", "M = Ul.T @ SW @ Vl", "M = (Ul.T @ SW @ Vl).T"),
    ("Sigma^{-1} dropped", "B = M / sl[:, None]", "B = M"),
    ("Sigma^{-1} on the wrong side", "B = M / sl[:, None]", "B = M / sl[None, :]"),
    ("SU updated from SAV", "SU_new = SW @ P", "SU_new = SAW @ P"),
    ("SAU updated from SV", "SAU_new = SAW @ P", "SAU_new = SW @ P"),
    ("U update shifted by one column", "U_new = np.hstack([U, V[:, :jf]]) @ P",
     "U_new = np.hstack([U, V[:, 1:jf + 1]]) @ P"),
    ("x_tilde from shifted columns", "x_tilde = np.hstack([U, V[:, :j + 1]]) @ y",
     "x_tilde = np.hstack([U, V[:, 1:j + 2]]) @ y"),
    ("sketch of r0 not normalised into SV", "SV[:, 0] = Sr0 / beta", "SV[:, 0] = Sr0"),
    ("exact variant keeps the old SAU", "SAU = S.apply_cols(csr_matmat(A, U))\n        res = solve(",
     "pass\n        res = solve("),
    ("missing SAU sketch when not provided", "SAU = S.apply_cols(csr_matmat(A, U))\n            matvecs",
     "SAU = S.apply_cols(U)\n            matvecs"),
    ("matvec drops the last entry of each row", "weights=A.val * x[A.col]",
     "weights=A.val * x[A.col] * (np.diff(np.r_[_row_index(A), A.n]) == 0)"),
]


def load_mutant(module, old, new):
    src = inspect.getsource(module)
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new, 1)
    mod = types.ModuleType(module.__name__ + "_mutant")
    mod.__dict__["__name__"] = module.__name__ + "_mutant"
    exec(compile(mutated, module.__file__ + "<mutant>", "exec"), mod.__dict__)
    return mod


def pins_catch(mod, pins):
    for pin in pins:
        try:
            with np.errstate(all="ignore"):
                pin(mod)
        except Exception:  # noqa: BLE001 - an assertion or a crash both mean "caught"
            return True
    return False


@pytest.mark.parametrize("name,old,new", SDR_MUTATIONS, ids=[m[0] for m in SDR_MUTATIONS])
def test_sdr_mutation_is_caught(name, old, new):
    mod = load_mutant(sdr, old, new)
    assert pins_catch(mod, P.ALL_PINS), f"no pin caught: {name}"


PART_MUTATIONS = [
    ("a conjugate pair split at the k-th eigenvalue", "        if mu[i].imag != 0.0:\n            for j in order:",
     "        if False:\n            for j in order:"),
    ("ties broken by the smaller real part", "np.lexsort((idx, -mu.real, -np.abs(mu)))",
     "np.lexsort((idx, mu.real, -np.abs(mu)))"),
    ("a complex pair contributes its real part only", "            cols.append(Y[:, i].imag)\n", ""),
    ("rank threshold from the smallest singular value", "sig > sig[0] * d * EPS", "sig > sig[-1] * d * EPS"),
    ("back substitution skips the last unknown", "R[i, i + 1:] @ y[i + 1:]", "R[i, i + 1:-1] @ y[i + 1:-1]"),
    ("least squares with R^T R in place of R", "y = back_substitute(R, Q.T @ Sr0)",
     "y = back_substitute(np.triu(R.T @ R), Q.T @ Sr0)"),
    ("a lucky breakdown does not end the cycle", "            if breakdown:\n                jf = j + 1\n                break",
     "            pass"),
    ("a lucky breakdown does not force the check", "if sres < tol / safety or j == m - 1 or breakdown:",
     "if sres < tol / safety or j == m - 1:"),
]


@pytest.mark.parametrize("name,old,new", PART_MUTATIONS, ids=[m[0] for m in PART_MUTATIONS])
def test_part_mutation_is_caught(name, old, new):
    import test_oracle_parts as T
    mod = load_mutant(sdr, old, new)
    assert pins_catch(mod, T.PART_PINS), f"no pin caught: {name}"


SKETCH_MUTATIONS = [
    ("sign from bit 1", "(w & np.uint64(1)) == 0", "(w & np.uint64(2)) == 0"),
    ("Floyd range off by one", "j = s - zeta + q", "j = s - zeta + q - 1"),
    ("Floyd keeps duplicates", "rows[:, q] = np.where(taken, j, t)", "rows[:, q] = t"),
    ("counter without the +1", "(c + np.uint64(1)) * GAMMA", "c * GAMMA"),
    ("mix64 wrong shift", "z ^ (z >> np.uint64(27))", "z ^ (z >> np.uint64(28))"),
    ("missing 1/sqrt(zeta)", "return y * self.scale", "return y"),
]


def _sketch_pins(mod):
    import test_oracle_sketch as T
    saved = {k: getattr(T, k) for k in ("sketch_indices", "splitmix64_at", "SparseSign")}
    try:
        T.sketch_indices, T.splitmix64_at, T.SparseSign = mod.sketch_indices, mod.splitmix64_at, mod.SparseSign
        fns = [T.test_splitmix64_known_answers, T.test_golden_table_matches, T.test_apply_matches_dense,
               T.test_subspace_embedding_distortion,
               lambda: T.test_floyd_rows_distinct_and_in_range(9, 8)]
        for f in fns:
            try:
                f()
            except Exception:  # noqa: BLE001
                return True
        return False
    finally:
        for k, v in saved.items():
            setattr(T, k, v)


@pytest.mark.parametrize("name,old,new", SKETCH_MUTATIONS, ids=[m[0] for m in SKETCH_MUTATIONS])
def test_sketch_mutation_is_caught(name, old, new):
    mod = load_mutant(sketch, old, new)
    assert _sketch_pins(mod), f"no pin caught: {name}"


# ---- the subsampled DCT (Section 6), pinned by its definition as a cosine sum
DCT_MUTATIONS = [
    ("DCT type III in place of II", "type=2", "type=3"),
    ("random signs dropped", "self.signs * x", "x"),
    ("scale sqrt(s / N)", "self.scale = np.sqrt(n / s)", "self.scale = np.sqrt(s / n)"),
    ("unnormalised DCT", 'norm="ortho"', 'norm="backward"'),
]


@pytest.mark.parametrize("name,old,new", DCT_MUTATIONS, ids=[m[0] for m in DCT_MUTATIONS])
def test_dct_mutation_is_caught(name, old, new, monkeypatch):
    import test_oracle_sketch as T
    mod = load_mutant(sketch, old, new)
    monkeypatch.setattr(sketch, "SubsampledDCT", mod.SubsampledDCT)  # the pin imports it from oracle.sketch
    assert pins_catch(mod, [lambda _m: T.test_subsampled_dct_definition_and_embedding()]), f"no pin caught: {name}"


# ---- the rank rule for an installed SAU and the stale-SAU rule (Section 3.6)
STALE_MUTATIONS = [
    ("rank threshold without the factor s", "<= s * EPS * maxn", "<= EPS * maxn"),
    ("rank test on the last pivot only", "np.any(np.abs(np.diag(R)) <= s * EPS * maxn)",
     "np.abs(R[-1, -1]) <= s * EPS * maxn"),
    ("non-finite SAU passes the rank test", "    if not np.all(np.isfinite(SAU)):\n        return True\n", ""),
    ("column norms taken over rows", "np.linalg.norm(SAU, axis=0)", "np.linalg.norm(SAU, axis=1)"),
    ("stale test with the ratio inverted", "c.checks[-1][2] > STALE_RATIO * c.checks[-1][1]",
     "c.checks[-1][1] > STALE_RATIO * c.checks[-1][2]"),
    ("stale refresh keeps the old SAU",
     "SAU = S.apply_cols(csr_matmat(A, U))\n            matvecs += U.shape[1]\n            refreshes += 1",
     "matvecs += U.shape[1]\n            refreshes += 1"),
]


def _stale_pins(mod):
    import test_oracle_stale as T
    saved = T.O
    try:
        T.O = mod
        return pins_catch(mod, [lambda _m: T.test_rank_rule_closed_forms(),
                                lambda _m: T.test_stale_rule_silent_on_exact_variant(30),
                                lambda _m: T.test_stale_rule_rescues_inexact_variant()])
    finally:
        T.O = saved


@pytest.mark.parametrize("name,old,new", STALE_MUTATIONS, ids=[m[0] for m in STALE_MUTATIONS])
def test_stale_mutation_is_caught(name, old, new):
    assert _stale_pins(load_mutant(sdr, old, new)), f"no pin caught: {name}"


# ---- the Givens-sine estimator (Section 4.5; Section 5, the augmented cycle)
GIVENS_MUTATIONS = [
    ("sine reported from the cosine", "sines.append(abs(s))", "sines.append(abs(c))"),
    ("earlier rotations not applied to the new column",
     "            Gr[k + i, col], Gr[k + i + 1, col] = c * a + s * b, -s * a + c * b\n", "            pass\n"),
    ("right-hand side from the column before", "g = beta * R[:, k].copy()", "g = beta * R[:, k - 1].copy()"),
    ("G without the Hessenberg block", "B[k:, k:] = H[:j + 1, :j]", "B[k:, k:] = np.eye(j + 1, j)"),
    ("rotation normalised by |a| + |b|", "r = float(np.hypot(a, b))", "r = float(abs(a) + abs(b))"),
]


def _givens_pins(mod):
    import test_oracle_givens as T
    saved = T.G
    try:
        T.G = mod
        return pins_catch(mod, [lambda _m: T.test_estimator_sres_equals_householder_least_squares(),
                                lambda _m: T.test_identity_sketch_gives_textbook_gmres_sines(),
                                lambda _m: T.test_sines_are_sketched_subspace_angles(),
                                lambda _m: T.test_corollary_bound_on_true_residuals()])
    finally:
        T.G = saved


@pytest.mark.parametrize("name,old,new", GIVENS_MUTATIONS, ids=[m[0] for m in GIVENS_MUTATIONS])
def test_givens_mutation_is_caught(name, old, new):
    from oracle import givens
    assert _givens_pins(load_mutant(givens, old, new)), f"no pin caught: {name}"
