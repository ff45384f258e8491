"""Pins for the oracle's sparse-sign embedding (Section 3, eq. (sketch)).

The hash is pinned by SplitMix64's published known-answer outputs, Floyd's
sampling by its defining properties, and the operator as a whole by the
subspace-embedding distortion it must show."""
import json
import os

import numpy as np
import pytest

from oracle.sketch import SparseSign, sketch_indices, splitmix64_at

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sketch_indices.json")


def test_splitmix64_known_answers():
    # Outputs of the reference SplitMix64 generator (Steele, Lea & Flood 2014;
    # the public splitmix64.c of Vigna) for seeds 0 and 1234567.
    assert [int(v) for v in splitmix64_at(0, np.arange(4))] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [int(v) for v in splitmix64_at(1234567, np.arange(5))] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


@pytest.mark.parametrize("s,zeta", [(120, 8), (480, 8), (100, 8), (9, 8), (8, 8), (5, 1)])
def test_floyd_rows_distinct_and_in_range(s, zeta):
    rows, signs = sketch_indices(231114206, s, zeta, np.arange(20000))
    assert rows.min() >= 0 and rows.max() < s
    srt = np.sort(rows, axis=1)
    assert np.all(np.diff(srt, axis=1) > 0), "rows of a column must be distinct"
    assert set(np.unique(signs)) <= {-1, 1}
    if s == zeta:  # every row used exactly once
        assert np.all(srt == np.arange(s))


def test_floyd_uniform_subsets_tiny():
    # s = 5, zeta = 2: Floyd's algorithm yields each of the 10 subsets with
    # probability 1/10 (Bentley & Floyd 1987).  Chi-square with 9 dof.
    n = 200000
    rows, _ = sketch_indices(7, 5, 2, np.arange(n))
    key = np.sort(rows, axis=1) @ np.array([5, 1])
    counts = np.bincount(key, minlength=25)
    subsets = [a * 5 + b for a in range(5) for b in range(a + 1, 5)]
    obs = counts[subsets]
    assert obs.sum() == n
    exp = n / 10
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 33.7  # p ~ 1e-4 for 9 dof


def test_row_load_and_sign_balance():
    n, s, zeta = 200000, 120, 8
    rows, signs = sketch_indices(231114206, s, zeta, np.arange(n))
    load = np.bincount(rows.ravel(), minlength=s)
    exp = n * zeta / s
    chi2 = ((load - exp) ** 2 / exp).sum()
    assert chi2 < 200  # 119 dof: mean 119, sd ~15.4
    frac = (signs > 0).mean()
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(signs.size)


def test_apply_matches_dense():
    S = SparseSign(3, 300, 40, 8)
    x = np.random.default_rng(0).standard_normal(300)
    D = S.dense()
    assert np.allclose(S.apply(x), D @ x, rtol=0, atol=1e-13)
    # every column has zeta entries of magnitude 1/sqrt(zeta)
    assert np.all((np.abs(D) > 0).sum(axis=0) == 8)
    assert np.allclose(np.abs(D[D != 0]), 1 / np.sqrt(8))


def test_subspace_embedding_distortion():
    # Section 3, eq. (sketch): for V with orthonormal columns the singular values
    # of S V lie in [sqrt(1-eps), sqrt(1+eps)].  For s = 2d a Gaussian embedding
    # gives singular values near [1 - sqrt(d/s), 1 + sqrt(d/s)]; a sparse-sign
    # embedding should stay inside that band widened by 10 %.
    N, d, s, zeta = 4096, 60, 120, 8
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((N, d)))
    lo, hi = 1 - np.sqrt(d / s), 1 + np.sqrt(d / s)
    eps_seen = []
    for seed in range(20):
        S = SparseSign(seed, N, s, zeta)
        sv = np.linalg.svd(S.apply_cols(Q), compute_uv=False)
        assert sv.min() > 0.9 * lo and sv.max() < 1.1 * hi
        eps_seen.append(1 - sv.min() ** 2)
    # the lower side of eq. (sketch) needs eps < 1: S must be injective on span(V)
    assert max(eps_seen) < 1.0
    # with s = 8 d the embedding must be much tighter
    S = SparseSign(5, N, 480, 8)
    sv = np.linalg.svd(S.apply_cols(Q), compute_uv=False)
    assert sv.min() > 0.55 and sv.max() < 1.45


def test_subsampled_dct_definition_and_embedding():
    """S = sqrt(N/s) P F E (Section 6): against the DCT-II written out as its
    cosine sum, E ||S x||^2 = ||x||^2 over the draws, and the distortion band of
    the sparse sign above."""
    from oracle.sketch import SubsampledDCT
    n, s = 64, 16
    S = SubsampledDCT(7, n, s)
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    C = np.sqrt(2.0 / n) * np.cos(np.pi * (2 * j + 1) * k / (2 * n))
    C[0, :] /= np.sqrt(2.0)  # orthonormal DCT-II
    ref = np.sqrt(n / s) * C[S.rows] * S.signs[None, :]
    assert np.allclose(S.dense(), ref, rtol=0, atol=1e-13)
    assert len(set(S.rows.tolist())) == s and S.rows.min() >= 0 and S.rows.max() < n
    x = np.random.default_rng(2).standard_normal(n)
    mean_sq = np.mean([np.sum(SubsampledDCT(sd, n, s).apply(x) ** 2) for sd in range(400)])
    assert mean_sq == pytest.approx(np.sum(x ** 2), rel=0.05)
    N, d, s2 = 4096, 60, 120
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((N, d)))
    lo, hi = 1 - np.sqrt(d / s2), 1 + np.sqrt(d / s2)
    for sd in range(10):
        sv = np.linalg.svd(SubsampledDCT(sd, N, s2).apply_cols(Q), compute_uv=False)
        assert sv.min() > 0.9 * lo and sv.max() < 1.1 * hi


def test_golden_table_matches():
    with open(GOLDEN) as f:
        g = json.load(f)
    for case in g["cases"]:
        rows, signs = sketch_indices(case["seed"], case["s"], case["zeta"], np.arange(case["ncols"]))
        assert rows.tolist() == case["rows"]
        assert signs.tolist() == case["signs"]
