// Internal definitions shared by the GMRES-SDR kernels and the host driver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sdr {

constexpr int M_MAX = 128;   // Krylov columns per cycle
constexpr int K_MAX = 32;    // recycle columns (k + 1)
constexpr int D_MAX = M_MAX + K_MAX;  // columns of SAW
constexpr int S_MAX = 768;   // sketch rows (the paper's experiments use s = 640)
constexpr int T_MAX = 4;     // Arnoldi truncation window
constexpr int ZETA_MAX = 32;
constexpr int PTR_STRIDE = S_MAX + 8;  // per-tile row-pointer stride (16-byte multiple)
constexpr int TILE_R = 1024; // rows per sketch tile (zeta*TILE_R < 65536 for uint16 offsets)
constexpr int NPART = 8;     // doubles of per-CTA partial results
constexpr int HIST_MAX = 1 << 15;  // logged Arnoldi steps per solve
constexpr int LOG_MAX = 512;       // logged cycles per solve

// Control block in device memory: the state that decides the cycle's control
// flow (Algorithm 1 residual control) without a host round trip per step.
struct Ctl {
  double tol, bnorm, bmax, anorm_inf;
  double safety, safety0, res, beta, sres;
  int kh;         // recycle columns used by the current cycle
  int done;       // current cycle finished (converged or forced end)
  int converged;  // true residual below tol
  int check;      // a true-residual check is due at the current step
  int jf;         // Krylov columns built when the cycle stopped
  int breakdown;
  int rankfail;
  int nchecks;
  int step;       // steps completed in the current cycle
  int acc_top;    // window top of the Arnoldi-vector sketch accumulators
  int accR_top;   // window top of the residual sketch accumulators
  int accG_top;   // window top of the general-purpose sketch accumulators
  int force_svd;  // test switch: always take the truncated-SVD path
  int ell, kprime, svd_path;
  int svd_sweeps; // Jacobi sweeps of the last truncated-SVD path
  int hist_n;     // logged steps so far in this solve
  int log_n;      // logged cycles so far in this solve
  int matvecs, sketches;
  int persist_safety;
  unsigned int counter;   // last-CTA counter for grid reductions on the Arnoldi stream
  unsigned int counter2;  // the same for the reductions of the dense (control) stream
  int jstop;      // jf of the check that ended the cycle (large while it runs)
  int bd_dense;   // the dense step of the current column saw H(j+1, j) = 0
  double alpha[M_MAX + 2];                // 1 / ||v_hat_c||
  int vtop[M_MAX + 2];                    // window top for the sketch of v_hat_c
  unsigned long long vmax[M_MAX + 2];     // bits of max |v_hat_c|
  unsigned long long wmax, xmax, rmax;    // bits of max |w|, |x_trial|, |r|
  unsigned long long umax[2][K_MAX];      // bits of max |U(:, l)| of each recycle buffer
  double hband[M_MAX][T_MAX + 1];         // H(i, j), i = j-t+1 .. j+1 at index i-(j-t+1)
  double gram[M_MAX + 2][T_MAX];          // v_hat_c . v_hat_{c-1-d}, d = 0..t-2
  double coef[T_MAX + 1];                 // a_0 (w) and a_1.. (window) for the update
  double hnext_sq;                        // ||v_hat_{j+1}||^2 (reduced in the dense step)
  int rank_sau;                           // the last installed SAU is numerically rank-deficient
  int tc_error;                           // a bounded wait of the tensor-core recycle kernel ran out
};

// The Arnoldi kernels of step j run while the dense step and the true-residual
// check of earlier columns run on a second stream.  The Arnoldi stream waits
// for the control work of column j - SPEC_LAG before step j, so a check that
// stopped the cycle at jf <= j - SPEC_LAG + 1 is final when step j starts, and
// any check still running can only set a larger jf: every CTA of a step sees
// the same answer.  Steps past the stop compute columns that nothing reads.
// Five: the control stream's time per column varies (real checks), and a
// shorter lag stalls the Arnoldi stream behind it; a longer one computes more
// steps past a converged check.
constexpr int SPEC_LAG = 5;
// Words of the per-cycle block that holds the column accumulators and the tile counters.
// Layout: the column accumulators, the tile counters ((M_MAX + 2) ints), and
// the window-dot accumulators of the Arnoldi SpMV (128 bits per step and dot).
constexpr size_t CYCLE_SCRATCH_WORDS = (size_t)(M_MAX + 2) * 2 * S_MAX + (M_MAX + 2) + (size_t)(M_MAX + 2) * T_MAX * 2;
__device__ __forceinline__ bool arnoldi_stopped(const Ctl* c, int j) { return c->jstop <= j - SPEC_LAG + 1; }

// Per-cycle log entry kept on the device, mirrored by sdr_cycle_log.
struct CycleLog {
  int steps, checks, converged, ell, kprime, kh, flags, svd_sweeps;
  double res, sres, safety;
};

// Device workspace: pointers and sizes, passed by value to kernels.
struct WS {
  int64_t n;        // current system size
  int64_t ldv;      // leading dimension of tall arrays (n_max rounded up to a multiple of 32)
  int m, k, t, s, zeta, kmax, dmax;
  int recycle_int;  // 1: the recycle product on the integer pipe instead of the tensor cores
  // sketch family: 0 the sparse sign (hash-defined, zeta nonzeros per column);
  // 1 the subsampled randomised DCT of the paper's experiments (Section 6),
  // S = sqrt(n/s) P F E, defined for one system size dct_n
  int sketch_kind;
  int64_t dct_n;
  const signed char* dct_sign;  // E: n random signs (+1 / -1)
  const int* dct_k;             // P: the s selected DCT-II frequencies
  const double* dct_cos;        // cos(pi m / (2n)), m = 0 .. n
  const double* dct_scale;      // per row: sqrt(n/s) alpha_k (alpha_0 = 1/sqrt(n), else sqrt(2/n))
  uint64_t seed;
  double inv_sqrt_zeta;
  int win_bits;     // log2 bound on terms per sketch row (window headroom)
  // tall arrays (n_max rows) of the solver's storage type (double, or float
  // for the refined form's inner solver); kernels cast them to that type
  void* Vs;         // columns 1..m of V (column c at Vs + (c-1)*ldv); column 0 is the residual
  void* R[2];       // residual buffers
  void* Wv;         // SpMV output w
  void* Xw;         // workspace iterate
  void* U[2];       // recycle bases, kmax columns each
  // sketch tables
  const uint16_t* sk_ent;  // per tile: zeta*TILE_R entries (offset | sign<<15)
  const uint16_t* sk_ptr;  // per tile: s+1 row pointers
  int ntiles;
  // reductions
  double* part;             // [grid_max][NPART]
  double* part2;            // [grid_max][NPART] partials of the Arnoldi update
  unsigned long long* acc;  // 128-bit accumulators, acc[2*i] = lo, acc[2*i+1] = hi
  unsigned long long* accV; // one accumulator block (2 * S_MAX words) per basis column c = 0 .. M_MAX+1
  int* tctr;                // per-step tile counters of the SpMV (dynamic tile scheduling), M_MAX+2
  double* part3;            // [grid_max][NPART] partials of the control-stream reductions
  unsigned long long* dacc; // [M_MAX + 2][T_MAX][2] window dots of step j, fixed point (in the cycle scratch)
  int grid_max;
  // small dense (column-major)
  double* SV;    // s x (m+1)
  double* SAV;   // s x m
  double* SU[2]; // s x kmax
  double* SAU[2];
  double* Y;     // s x dmax Householder vectors
  unsigned long long* Yq;  // s x dmax fixed-point copy of Y (|Y| <= 1, unit 2^-50)
  unsigned long long* Tq;  // dmax x dmax fixed-point copy of T, scaled per column
  int* texp;     // dmax: frexp exponent of each T column's scale
  double* T;     // dmax x dmax
  double* Rf;    // dmax x dmax
  double* tau;   // dmax
  double* z;     // s: Q^T S r0 as reflectors are added
  double* Sr0;   // s
  double* ytil;  // dmax
  double* P;     // dmax x kmax: recycle coefficients (V rows scaled by alpha)
  unsigned long long* Pq;  // D_MAX x K_MAX fixed-point P'' (Q52 bits) for the tall update
  int* Pexp;     // K_MAX: exponent of each P'' column's scale
  unsigned long long* ytq; // D_MAX fixed-point y'' for the check GEMV
  int* yexp;     // [0]: exponent of y'' scale
  double* dscr;  // dense scratch for the cycle-end kernel
  double* hist;  // HIST_MAX sres values
  double* hist_givens;  // 2 x HIST_MAX: Givens sine and cosine of each step (Section 4.5, Section 5)
  CycleLog* log; // LOG_MAX entries
  Ctl* ctl;
};

// ---------------------------------------------------------------------------
// Hash-defined sparse-sign embedding (same definition as the oracle, written
// independently): word(c, q) = SplitMix64 output number c*zeta + q for the
// seed; rows by Floyd's sampling; sign from bit 0.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t splitmix_word(uint64_t seed, uint64_t counter) {
  return mix64(seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull);
}

// Rows (distinct, in [0, s)) and signs (+1/-1) of sketch column c.
__host__ __device__ inline void sketch_column(uint64_t seed, int s, int zeta, uint64_t c,
                                              int* rows, int* signs) {
  for (int q = 0; q < zeta; ++q) {
    uint64_t w = splitmix_word(seed, c * (uint64_t)zeta + (uint64_t)q);
    uint32_t j = (uint32_t)(s - zeta + q);
    uint32_t hi = (uint32_t)(w >> 32);
    uint32_t t = (uint32_t)(((uint64_t)hi * (uint64_t)(j + 1)) >> 32);
    bool taken = false;
    for (int p = 0; p < q; ++p) taken |= (rows[p] == (int)t);
    rows[q] = taken ? (int)j : (int)t;
    signs[q] = (w & 1ull) ? -1 : 1;
  }
}

// ---------------------------------------------------------------------------
// Fixed-point helpers for the exact sketch accumulation.
// ---------------------------------------------------------------------------
// Bits of |x| (sign cleared); unsigned order of these bits is the order of |x|.
__device__ inline unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Biased exponent field of a non-negative double given by its bits.
__host__ __device__ inline int bexp_of_bits(unsigned long long b) { return (int)((b >> 52) & 0x7FF); }

// Quantise x to round(x * 2^(51 - e)) where 2^(e-1) <= maxabs < 2^e has biased
// exponent field emax (so e = emax - 1022).  |result| <= 2^51.  Integer-only.
__device__ inline long long quantize_fixed(double x, int emax) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;  // zero or subnormal: below the quantum
  unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  // x = mant * 2^(ex - 1075); q = x * 2^(51 - (emax - 1022)) = mant * 2^(ex - emax - 2)
  int sh = emax + 2 - ex;  // >= 2 because ex <= emax
  if (sh >= 63) return 0;
  unsigned long long q = (mant + (1ull << (sh - 1))) >> sh;
  return (b >> 63) ? -(long long)q : (long long)q;
}

// 128-bit two's-complement add of a sign-extended 64-bit value shifted left by sh.
__device__ inline void add_shifted128(unsigned long long& lo, unsigned long long& hi, long long v, int sh) {
  if (v == 0) return;
  unsigned long long vlo, vhi;
  if (sh >= 64) {
    vlo = 0ull;
    vhi = (unsigned long long)(v << (sh - 64));
  } else if (sh > 0) {
    vlo = (unsigned long long)v << sh;
    vhi = (unsigned long long)(v >> (64 - sh));
  } else if (sh == 0) {
    vlo = (unsigned long long)v;
    vhi = (unsigned long long)(v >> 63);
  } else {
    int r = -sh;
    if (r >= 63) return;
    long long rv = (v + (1ll << (r - 1))) >> r;  // round to nearest
    vlo = (unsigned long long)rv;
    vhi = (unsigned long long)(rv >> 63);
  }
  unsigned long long nlo = lo + vlo;
  hi += vhi + (nlo < lo ? 1ull : 0ull);
  lo = nlo;
}

// Atomically add a 128-bit value into acc[0] (lo), acc[1] (hi).  Integer
// addition is associative, so the final sum does not depend on the order.
__device__ inline void atomic_add128(unsigned long long* acc, unsigned long long lo, unsigned long long hi) {
  if (lo == 0ull && hi == 0ull) return;
  unsigned long long old = atomicAdd(acc, lo);
  unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(acc + 1, hi + carry);
}

// Signed 128-bit (hi:lo) times 2^scale_exp, rounded to double.
__device__ inline double int128_to_double(unsigned long long lo, unsigned long long hi, int scale_exp) {
  bool neg = (long long)hi < 0;
  if (neg) {  // negate
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  double d = (double)hi * 18446744073709551616.0 + (double)lo;
  d = ldexp(d, scale_exp);
  return neg ? -d : d;
}

// Window for a sketch of a vector whose entries are bounded by `bound`: the
// 128-bit accumulator counts in units of 2^(top - 126), top = exponent of
// bound + log2(number of summed terms) + 2.
__host__ __device__ inline int window_top(double bound, int win_bits) {
  int e;
  frexp(bound > 0.0 ? bound : 1e-300, &e);
  return e + win_bits + 2;
}

// Add a double d to a 128-bit accumulator counting in units of 2^(top - 126)
// (rounded to the unit; |d| < 2^top by the choice of the window).
__device__ inline void add_double128(unsigned long long& lo, unsigned long long& hi, double d, int top) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) return;  // zero (subnormals are below any unit here) or not finite
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  add_shifted128(lo, hi, (b >> 63) ? -mant : mant, (ex - 1075) - (top - 126));
}

// ---------------------------------------------------------------------------
// Sketch tiles.
// ---------------------------------------------------------------------------
__host__ __device__ inline int sketch_tile_rows(int zeta) {
  int r = 32768 / (zeta > 0 ? zeta : 1);
  if (r > TILE_R) r = TILE_R;
  r = (r / 512) * 512;
  return r < 512 ? 512 : r;
}
inline size_t sketch_smem_bytes(int zeta) {
  int tileR = sketch_tile_rows(zeta);
  return (size_t)tileR * 8 + (size_t)tileR * zeta * 2 + (S_MAX + 16) * 2;
}
constexpr int SK_THREADS = 256;              // threads of the tile-sketch kernels
constexpr int SK_RPT = S_MAX / SK_THREADS;   // sketch rows per thread
constexpr int SK_RPT_SMALL = 2;              // the same for s <= 2 SK_THREADS (the SpMV's lighter instance)

// ---------------------------------------------------------------------------
// Block-level helpers.
// ---------------------------------------------------------------------------
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline unsigned long long warp_max_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Sum over the block in a fixed order (deterministic).  `red` needs
// blockDim.x/32 doubles of shared memory.  All threads receive the result.
__device__ inline double block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < nw ? red[lane] : 0.0;
    r = warp_sum(r);
    if (lane == 0) red[0] = r;
  }
  __syncthreads();
  r = red[0];
  __syncthreads();
  return r;
}

// Block sum with one FP64 add per value staged: every thread stores its value,
// the first warp adds blockDim/32 values per lane and then reduces across lanes
// (about a dozen FP64 warp instructions for 256 threads instead of ~45 for a
// shuffle tree per warp).  buf needs blockDim.x doubles.  Fixed order.
__device__ inline double block_sum_lean(double v, double* buf) {
  __syncthreads();
  buf[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int i = threadIdx.x; i < blockDim.x; i += 32) a += buf[i];
    a = warp_sum(a);
    if (threadIdx.x == 0) buf[0] = a;
  }
  __syncthreads();
  const double r = buf[0];
  __syncthreads();
  return r;
}

__device__ inline unsigned long long block_max_u64(unsigned long long v, unsigned long long* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max_u64(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    unsigned long long r = lane < nw ? red[lane] : 0ull;
    r = warp_max_u64(r);
    if (lane == 0) red[0] = r;
  }
  __syncthreads();
  unsigned long long r = red[0];
  __syncthreads();
  return r;
}

// Sketch of one tile: the tile's index lists (tileR*zeta offsets and s+1 row
// pointers) are copied to shared memory with cp.async (16-byte pieces) so the
// copy overlaps the caller's computation of the tile's values.
__device__ inline void tile_sketch_prefetch(const WS& ws, int tileR, int tile, uint16_t* ent_s, uint16_t* ptr_s) {
  const char* src = (const char*)(ws.sk_ent + (int64_t)tile * tileR * ws.zeta);
  const int nvec = (tileR * ws.zeta) / 8;  // 16-byte pieces
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(ent_s + 8 * i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(src + 16 * (int64_t)i));
  }
  const char* psrc = (const char*)(ws.sk_ptr + (int64_t)tile * PTR_STRIDE);
  // S_MAX + 1 uint16 rounded down to whole 16-byte pieces, the tail by plain loads
  const int pvec = ((ws.s + 1) * 2) / 16;
  for (int i = threadIdx.x; i < pvec; i += blockDim.x) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(ptr_s + 8 * i);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(psrc + 16 * (int64_t)i));
  }
  asm volatile("cp.async.commit_group;\n" ::);
  const uint16_t* pp = ws.sk_ptr + (int64_t)tile * PTR_STRIDE;
  for (int i = pvec * 8 + threadIdx.x; i <= ws.s; i += blockDim.x) ptr_s[i] = pp[i];
}

// Add the tile's contribution S_tile x_tile to the 128-bit accumulators of the
// sketch rows this thread owns (rows threadIdx.x + q * blockDim.x, q < RPT).
// vals holds the tile's values (tileR doubles, zero beyond ncols) and is
// overwritten; the index lists must have been prefetched.  All threads of the
// block must call it.
template <int RPT>
__device__ inline void tile_sketch_accumulate(const WS& ws, int ncols, double* vals, const uint16_t* ent_s,
                                              const uint16_t* ptr_s, unsigned long long* red, int top,
                                              unsigned long long* lo, unsigned long long* hi) {
  asm volatile("cp.async.wait_all;\n" ::);
  unsigned long long mb = 0ull;
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
    const unsigned long long b = abs_bits(vals[i]);
    mb = b > mb ? b : mb;
  }
  mb = block_max_u64(mb, red);  // synchronises the block (also publishes the prefetch)
  const int emax = bexp_of_bits(mb);
  if (emax == 0 || emax == 0x7FF) return;  // all zero, or non-finite (caught through the norms)
  long long* q = (long long*)vals;
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) q[i] = quantize_fixed(vals[i], emax);
  __syncthreads();
  const int sh = (emax - 1022) - 51 - (top - 126);  // tile unit 2^(e_t - 51) in window units
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int row = threadIdx.x + k * blockDim.x;
    if (row < ws.s) {
      long long a = 0;
      const int e0 = ptr_s[row], e1 = ptr_s[row + 1];
      for (int e = e0; e < e1; ++e) {
        const uint16_t c = ent_s[e];
        const long long v = q[c & 0x7FFF];
        a += (c & 0x8000) ? -v : v;
      }
      add_shifted128(lo[k], hi[k], a, sh);
    }
  }
  __syncthreads();
}

// The same for the subsampled randomised DCT (sketch_kind 1; Section 6): row r
// of S x is dct_scale[r] sum_i E_i x_i cos(pi (2i + 1) k_r / (2n)).  Each
// thread forms the tile's partial sum of each of its rows in FP64, in index
// order (so the result does not depend on the grid), and adds it to its
// 128-bit accumulators.  The cosine comes from the table of cos(pi m / (2n)),
// m = 0 .. n, by the symmetries of cos over [0, 4n).  vals holds the tile
// (zero beyond ncols) and is overwritten; all threads of the block call it.
template <int RPT>
__device__ inline void tile_dct_accumulate(const WS& ws, int64_t r0, int ncols, double* vals, int top,
                                           unsigned long long* lo, unsigned long long* hi) {
  __syncthreads();
  for (int i = threadIdx.x; i < ncols; i += blockDim.x)
    if (ws.dct_sign[r0 + i] < 0) vals[i] = -vals[i];
  __syncthreads();
  const unsigned int n = (unsigned int)ws.dct_n, n2 = 2u * n, n4 = 4u * n;  // n < 2^29 (checked on the host)
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int row = threadIdx.x + k * blockDim.x;
    if (row < ws.s) {
      const unsigned long long f = (unsigned long long)ws.dct_k[row];
      unsigned int m = (unsigned int)(((2ull * (unsigned long long)r0 + 1ull) * f) % n4);  // (2i + 1) f mod 4n
      const unsigned int step = (unsigned int)((2ull * f) % n4);
      double acc0 = 0.0, acc1 = 0.0;
      for (int i = 0; i < ncols; ++i) {
        const unsigned int a = m > n2 ? n4 - m : m;  // cos(pi a / 2n) = cos(pi m / 2n)
        const double cv = a > n ? -__ldg(ws.dct_cos + (n2 - a)) : __ldg(ws.dct_cos + a);
        if (i & 1)
          acc1 = fma(vals[i], cv, acc1);
        else
          acc0 = fma(vals[i], cv, acc0);
        m += step;
        if (m >= n4) m -= n4;
      }
      add_double128(lo[k], hi[k], (acc0 + acc1) * ws.dct_scale[row], top);
    }
  }
  __syncthreads();
}

}  // namespace sdr
