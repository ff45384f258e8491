"""Sparse-sign subspace embedding S, defined by a counter-based hash.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Section 3 (eq. (sketch)) asks for an s x N operator S that is an
epsilon-subspace embedding; the paper's experiments used a subsampled DCT.
This build uses a sparse-sign embedding: column c of S has exactly zeta
nonzeros, each +-1/sqrt(zeta), in zeta distinct rows.

Definition (bit-exact; the CUDA path implements the same definition on its
own):

  word(c, q)  = SplitMix64 output number c*zeta + q (0-based) of the generator
                seeded with `seed` (Steele, Lea & Flood, OOPSLA 2014), i.e.
                mix64(seed + (c*zeta + q + 1) * 0x9E3779B97F4A7C15 mod 2^64).
  rows        = Floyd's algorithm (Bentley & Floyd, CACM 1987) for a uniform
                zeta-subset of {0..s-1}: for q = 0..zeta-1 with j = s-zeta+q,
                t = floor(hi32(word(c,q)) * (j+1) / 2^32); the row of slot q is
                t unless t is already a row of an earlier slot, then it is j.
  sign of q   = +1 if bit 0 of word(c,q) is 0, else -1.
  S[row, c]   = sign / sqrt(zeta).
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (wrapping uint64 arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_at(seed: int, counter) -> np.ndarray:
    """Output number `counter` (0-based) of SplitMix64 seeded with `seed`."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
    return mix64(state)


def sketch_indices(seed: int, s: int, zeta: int, cols) -> tuple:
    """Rows (int32 [n, zeta]) and signs (int8 [n, zeta]) of the given columns."""
    if not 1 <= zeta <= s:
        raise ValueError("need 1 <= zeta <= s")
    cols = np.asarray(cols, dtype=np.uint64)
    n = cols.shape[0]
    rows = np.empty((n, zeta), dtype=np.int64)
    signs = np.empty((n, zeta), dtype=np.int8)
    base = cols * np.uint64(zeta)
    for q in range(zeta):
        w = splitmix64_at(seed, base + np.uint64(q))
        j = s - zeta + q
        t = ((w >> np.uint64(32)) * np.uint64(j + 1)) >> np.uint64(32)
        t = t.astype(np.int64)
        taken = np.zeros(n, dtype=bool)
        for p in range(q):
            taken |= rows[:, p] == t
        rows[:, q] = np.where(taken, j, t)
        signs[:, q] = np.where((w & np.uint64(1)) == 0, 1, -1).astype(np.int8)
    return rows.astype(np.int32), signs


class SparseSign:
    """S x for the hash-defined sparse-sign embedding (indices cached)."""

    def __init__(self, seed: int, n: int, s: int, zeta: int):
        self.seed, self.n, self.s, self.zeta = seed, n, s, zeta
        self.rows, self.signs = sketch_indices(seed, s, zeta, np.arange(n))
        self.scale = 1.0 / np.sqrt(float(zeta))

    def apply(self, x: np.ndarray) -> np.ndarray:
        """(S x)_r = (1/sqrt(zeta)) sum over (c, q) with row(c,q) = r of sign(c,q) x_c."""
        contrib = self.signs.astype(np.float64) * x[:, None]
        y = np.bincount(self.rows.ravel(), weights=contrib.ravel(), minlength=self.s)
        return y * self.scale

    def apply_cols(self, X: np.ndarray) -> np.ndarray:
        return np.stack([self.apply(X[:, i]) for i in range(X.shape[1])], axis=1) \
            if X.shape[1] else np.zeros((self.s, 0))

    def dense(self) -> np.ndarray:
        """The s x N matrix (small n only; for tests)."""
        D = np.zeros((self.s, self.n))
        for q in range(self.zeta):
            D[self.rows[:, q], np.arange(self.n)] += self.signs[:, q] * self.scale
        return D


class SubsampledDCT:
    """The sketch of the paper's experiments (Section 6, opening paragraph):
    S = sqrt(N / s) P F E with E a diagonal of random signs, F the orthonormal
    DCT (type II; scipy's transform serves as the library step) and P the
    selection of s distinct rows drawn uniformly at random.  E ||S x||^2 =
    ||x||^2.  The second sketch family, beside the sparse sign above: it runs
    the paper's experiments with the paper's operator.
    The random signs and rows come from numpy's PCG64 seeded [seed, n, s]."""

    def __init__(self, seed: int, n: int, s: int):
        g = np.random.default_rng([seed, n, s])
        self.seed, self.n, self.s = seed, n, s
        self.signs = g.choice(np.array([-1.0, 1.0]), n)
        self.rows = np.sort(g.choice(n, s, replace=False))
        self.scale = np.sqrt(n / s)

    def apply(self, x: np.ndarray) -> np.ndarray:
        import scipy.fft
        return self.scale * scipy.fft.dct(self.signs * x, type=2, norm="ortho")[self.rows]

    def apply_cols(self, X: np.ndarray) -> np.ndarray:
        return np.stack([self.apply(X[:, i]) for i in range(X.shape[1])], axis=1) \
            if X.shape[1] else np.zeros((self.s, 0))

    def dense(self) -> np.ndarray:
        """The s x N matrix (small n only; for tests)."""
        return self.apply_cols(np.eye(self.n))


class Identity:
    """S = I (s = N): reduces GMRES-SDR to unsketched augmented GMRES."""

    def __init__(self, n: int):
        self.n = self.s = n

    def apply(self, x):
        return np.array(x, dtype=np.float64, copy=True)

    def apply_cols(self, X):
        return np.array(X, dtype=np.float64, copy=True)

    def dense(self):
        return np.eye(self.n)
