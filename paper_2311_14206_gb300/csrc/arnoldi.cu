// Streaming kernels of one GMRES-SDR cycle (Algorithm 1), FP64.
//
//  k_spmv_dots     w = A v_j and the dots of w with the truncation window;
//                  the last CTA turns them into the MGS coefficients H(i, j).
//  k_update_sketch v_hat_{j+1} = w - sum_i H(i,j) v_i (truncated Arnoldi), its
//                  norm and window dots, and S v_hat_{j+1} (one sketch per step).
//  k_residual      r = b - A x with ||r|| and S r; applies the residual control
//                  of Section 3.4 when it serves a true-residual check.
//  k_check_gemv    x_trial = x + [U V] y_tilde.
//  k_recycle_gemm  U_new = [U V] P (recycle update, Section 3.5).
//
// Basis columns are stored unnormalised (v_hat); alpha_c = 1/||v_hat_c|| lives
// in the control block and is folded into every coefficient that touches a
// column, which saves a normalisation pass per step.
#include <type_traits>

#include "launch.cuh"
#include "eidot.cuh"

namespace sdr {

// Tall vectors (the basis, w, residuals, iterates, U) hold elements of type T:
// double for the FP64 solver, float for the FP32 inner solver of the refined
// form, whose SpMV, window dots and updates then also accumulate in FP32.
template <typename T>
struct Win {
  const T* v[T_MAX];  // v_hat_lo .. v_hat_j
  int lo, nw;
};

template <typename T> __device__ __forceinline__ const T* csr_val(const CsrDev& A);
template <> __device__ __forceinline__ const double* csr_val<double>(const CsrDev& A) { return A.val; }
template <> __device__ __forceinline__ const float* csr_val<float>(const CsrDev& A) { return A.val32; }

template <typename T>
__device__ inline T csr_row_dot(const CsrDev& A, const T* __restrict__ x, int64_t r) {
  const int32_t* __restrict__ rowptr = A.rowptr;
  const int32_t* __restrict__ col = A.col;
  const T* __restrict__ val = csr_val<T>(A);
  int p0 = rowptr[r], p1 = rowptr[r + 1];
  T y = 0;
  for (int p = p0; p < p1; ++p) y = fma(val[p], x[col[p]], y);
  return y;
}

// Two CSR rows at once (either may be absent): the column indices and values
// of both rows are loaded in chunks of seven before the gathers and the
// products, so a thread keeps two rows' worth of loads in flight.  Each row's
// sum is formed in column order exactly as in csr_row_dot.
template <typename T>
__device__ __forceinline__ void csr_row_pair(const CsrDev& A, const T* __restrict__ x, int64_t ra, bool va_,
                                             int64_t rb, bool vb_, T& ya, T& yb) {
  const int32_t* __restrict__ rp = A.rowptr;
  const int32_t* __restrict__ ci = A.col;
  const T* __restrict__ av = csr_val<T>(A);
  int a0 = va_ ? rp[ra] : 0, a1 = va_ ? rp[ra + 1] : 0;
  int b0 = vb_ ? rp[rb] : 0, b1 = vb_ ? rp[rb + 1] : 0;
  // a chunk of seven covers a 7-point stencil row in one pass (a masked FP64
  // instruction costs as much as a full one on this GPU)
  constexpr int U = 7;
  T sa = 0, sb = 0;
  while (a0 < a1 || b0 < b1) {
    int ca[U], cb[U];
    T pa[U], pb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ua = a0 + u < a1, ub = b0 + u < b1;
      ca[u] = ua ? ci[a0 + u] : -1;
      pa[u] = ua ? av[a0 + u] : (T)0;
      cb[u] = ub ? ci[b0 + u] : -1;
      pb[u] = ub ? av[b0 + u] : (T)0;
    }
    T xa[U], xb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      xa[u] = ca[u] >= 0 ? x[ca[u]] : (T)0;
      xb[u] = cb[u] >= 0 ? x[cb[u]] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (ca[u] >= 0) sa = fma(pa[u], xa[u], sa);
      if (cb[u] >= 0) sb = fma(pb[u], xb[u], sb);
    }
    a0 += U;
    b0 += U;
  }
  ya = sa;
  yb = sb;
}

// Last CTA of a grid: returns true in exactly one CTA after every CTA has
// published its partials (threadfence + counter; the counter is re-armed).
__device__ inline bool last_block(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return am_last;
}

// Fixed-order sum of part[b*NPART + k] over b < nb (all threads get it).
__device__ inline double reduce_parts(const double* part, int nb, int k, double* red) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b * NPART + k];
  return block_sum(v, red);
}
__device__ inline unsigned long long reduce_parts_max(const double* part, int nb, int k, unsigned long long* red) {
  unsigned long long v = 0ull;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    unsigned long long u = (unsigned long long)__double_as_longlong(part[b * NPART + k]);
    v = u > v ? u : v;
  }
  return block_max_u64(v, red);
}

// ---------------------------------------------------------------------------
// Solve start: ||b||, max|b|, max|x0|, ||A||_inf, tol.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_solve_init(WS ws, CsrDev A, const T* __restrict__ b, const T* __restrict__ x, double rel_tol,
                             int keep_logs) {
  __shared__ double red[32];
  __shared__ unsigned long long redu[32];
  double bb = 0.0;
  unsigned long long bm = 0ull, xm = 0ull, am = 0ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.n; r += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)b[r];
    bb = fma(v, v, bb);
    unsigned long long u = abs_bits(v);
    bm = u > bm ? u : bm;
    u = abs_bits((double)x[r]);
    xm = u > xm ? u : xm;
    double rs = 0.0;
    const T* __restrict__ av = csr_val<T>(A);
    for (int p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) rs += fabs((double)av[p]);
    u = abs_bits(rs);
    am = u > am ? u : am;
  }
  bb = block_sum(bb, red);
  bm = block_max_u64(bm, redu);
  xm = block_max_u64(xm, redu);
  am = block_max_u64(am, redu);
  if (threadIdx.x == 0) {
    double* pp = ws.part + blockIdx.x * NPART;
    pp[0] = bb;
    pp[1] = __longlong_as_double((long long)bm);
    pp[2] = __longlong_as_double((long long)xm);
    pp[3] = __longlong_as_double((long long)am);
  }
  Ctl* c = ws.ctl;
  if (last_block(&c->counter)) {
    double s = reduce_parts(ws.part, gridDim.x, 0, red);
    unsigned long long m1 = reduce_parts_max(ws.part, gridDim.x, 1, redu);
    unsigned long long m2 = reduce_parts_max(ws.part, gridDim.x, 2, redu);
    unsigned long long m3 = reduce_parts_max(ws.part, gridDim.x, 3, redu);
    if (threadIdx.x == 0) {
      c->bnorm = sqrt(s);
      c->tol = rel_tol * c->bnorm;
      c->bmax = __longlong_as_double((long long)m1);
      c->xmax = m2;
      c->anorm_inf = __longlong_as_double((long long)m3);
      if (!keep_logs) {  // a refinement's inner solve appends to the outer solve's logs and counts
        c->hist_n = 0;
        c->log_n = 0;
        c->matvecs = 0;
        c->sketches = 0;
      }
      c->done = 0;
      c->converged = 0;
      c->check = 0;
      c->safety = c->safety0;
    }
  }
}

static int grid_rows(int64_t n, int tpb, int gmax) {
  int64_t g = (n + tpb - 1) / tpb;
  if (g > gmax) g = gmax;
  return g < 1 ? 1 : (int)g;
}

template <typename T>
cudaError_t launch_solve_init_x(const WS& ws, CsrDev A, const T* b, const T* x, double rel_tol, cudaStream_t st,
                                bool keep_logs) {
  k_solve_init<T><<<grid_rows(A.n, 256, ws.grid_max), 256, 0, st>>>(ws, A, b, x, rel_tol, keep_logs ? 1 : 0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// True residual r = b - A x with ||r||, max|r| and S r (tile-fused).
// mode 0: unconditional (solve start).  mode 1: runs only when ctl->check and
// then applies Algorithm 1's residual control in the last CTA.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_residual(WS ws, CsrDev A, const T* __restrict__ b, const T* __restrict__ x,
                           T* __restrict__ rout, unsigned long long* accR, int j, int mode,
                           double* __restrict__ part, unsigned int* counter) {
  Ctl* c = ws.ctl;
  if (mode == 1 && !c->check) return;
  extern __shared__ unsigned char smem[];
  const int tileR = sketch_tile_rows(ws.zeta);
  double* vals = (double*)smem;
  uint16_t* ent_s = (uint16_t*)(vals + tileR);
  uint16_t* ptr_s = ent_s + tileR * ws.zeta;
  __shared__ unsigned long long redu[32];
  __shared__ double red[32];
  const double xm = __longlong_as_double((long long)c->xmax);
  const int top = window_top((c->bmax + c->anorm_inf * xm) * (1.0 + 1e-12), ws.win_bits);
  unsigned long long lo[SK_RPT], hi[SK_RPT], rm = 0ull;
#pragma unroll
  for (int k = 0; k < SK_RPT; ++k) lo[k] = hi[k] = 0ull;
  double nrm = 0.0;
  const int64_t n = A.n;
  const int ntiles = (int)((n + tileR - 1) / tileR);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * tileR;
    const int ncols = (int)(n - r0 < (int64_t)tileR ? n - r0 : (int64_t)tileR);
    if (!ws.sketch_kind) tile_sketch_prefetch(ws, tileR, tile, ent_s, ptr_s);
    for (int i = threadIdx.x; i < tileR; i += blockDim.x) {
      double v = 0.0;
      if (i < ncols) {
        int64_t r = r0 + i;
        const T vt = b[r] - csr_row_dot<T>(A, x, r);
        rout[r] = vt;
        v = (double)vt;
        nrm = fma(v, v, nrm);
        unsigned long long u = abs_bits(v);
        rm = u > rm ? u : rm;
      }
      vals[i] = v;
    }
    if (ws.sketch_kind)
      tile_dct_accumulate<SK_RPT>(ws, r0, ncols, vals, top, lo, hi);
    else
      tile_sketch_accumulate<SK_RPT>(ws, ncols, vals, ent_s, ptr_s, redu, top, lo, hi);
  }
#pragma unroll
  for (int k = 0; k < SK_RPT; ++k) {
    const int row = threadIdx.x + k * blockDim.x;
    if (row < ws.s) atomic_add128(accR + 2 * row, lo[k], hi[k]);
  }
  nrm = block_sum(nrm, red);
  rm = block_max_u64(rm, redu);
  if (threadIdx.x == 0) {
    part[blockIdx.x * NPART + 0] = nrm;
    part[blockIdx.x * NPART + 1] = __longlong_as_double((long long)rm);
  }
  if (last_block(counter)) {
    double s = reduce_parts(part, gridDim.x, 0, red);
    unsigned long long m = reduce_parts_max(part, gridDim.x, 1, redu);
    if (threadIdx.x == 0) {
      double res = sqrt(s);
      c->res = res;
      c->rmax = m;
      c->accR_top = top;
      atomicAdd(&c->matvecs, 1);
      atomicAdd(&c->sketches, 1);
      if (mode == 1) {
        c->nchecks += 1;
        c->check = 0;
        if (res < c->tol) {
          c->converged = 1;
          c->done = 1;
          c->jf = j + 1;
          c->jstop = j + 1;
        } else {
          c->safety = c->sres > 0.0 ? res / c->sres : c->safety;  // increase the safety factor
          if (j == ws.m - 1 || c->bd_dense) {
            c->done = 1;
            c->jf = j + 1;
            c->jstop = j + 1;
          }
        }
      } else {
        c->converged = res < c->tol ? 1 : 0;
      }
    }
  }
}

// Raise a kernel's dynamic shared-memory limit once per process.
static cudaError_t set_smem(const void* f, size_t sm, bool& done) {
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) done = true;
  return e;
}

static int grid_tiles(const WS& ws, int64_t n) {
  int tileR = sketch_tile_rows(ws.zeta);
  int ntiles = (int)((n + tileR - 1) / tileR);
  const int gmax = ws.grid_max / 2;  // four CTAs per SM
  int g = ntiles < gmax ? ntiles : gmax;
  return g < 1 ? 1 : g;
}

template <typename T>
cudaError_t launch_residual(const WS& ws, CsrDev A, const T* b, const T* x, T* rout,
                            unsigned long long* accR, int j, int mode, cudaStream_t st) {
  size_t sm = sketch_smem_bytes(ws.zeta);
  static bool attr = false;
  cudaError_t e = set_smem((const void*)k_residual<T>, sketch_smem_bytes(ZETA_MAX), attr);
  if (e != cudaSuccess) return e;
  // the check (mode 1) runs on the control stream beside the Arnoldi kernels:
  // it reduces through its own partials and counter
  double* part = mode == 1 ? ws.part3 : ws.part;
  unsigned int* counter = mode == 1 ? &ws.ctl->counter2 : &ws.ctl->counter;
  k_residual<T><<<grid_tiles(ws, A.n), SK_THREADS, sm, st>>>(ws, A, b, x, rout, accR, j, mode, part, counter);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Column j of the basis is finished by the first kernel that runs after the
// update which produced it: h(j, j-1) = ||v_hat_j||, alpha_j = 1/h, the window
// dots v_hat_j . v_hat_{j-1-d} and max |v_hat_j| are reduced from the update's
// per-CTA partials (fixed order).  Runs in one CTA.
// ---------------------------------------------------------------------------
__device__ void finish_column(const WS& ws, int j, int grid2, double* buf, unsigned long long* redu) {
  Ctl* c = ws.ctl;
  const int t = ws.t;
  double v = 0.0;
  for (int b = threadIdx.x; b < grid2; b += blockDim.x) v += ws.part2[b * NPART + 0];
  const double nrm = block_sum_lean(v, buf);
  double cross[T_MAX - 1];
#pragma unroll
  for (int d = 0; d < T_MAX - 1; ++d) {
    double cv = 0.0;
    if (d < t - 1) {
      for (int b = threadIdx.x; b < grid2; b += blockDim.x) cv += ws.part2[b * NPART + 1 + d];
      cv = block_sum_lean(cv, buf);
    }
    cross[d] = cv;
  }
  unsigned long long vm = 0ull;
  for (int b = threadIdx.x; b < grid2; b += blockDim.x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(ws.part2[b * NPART + T_MAX]);
    vm = u > vm ? u : vm;
  }
  vm = block_max_u64(vm, redu);
  if (threadIdx.x == 0) {
    const double h = sqrt(nrm);
    const bool bd = !(h > 0.0) || !isfinite(h);
    c->alpha[j] = bd ? 0.0 : 1.0 / h;
    c->vmax[j] = vm;
    for (int d = 0; d < t - 1; ++d) c->gram[j][d] = cross[d];
    c->hband[j - 1][t] = bd ? 0.0 : h;  // H(j, j-1)
    if (bd) c->breakdown = 1;
  }
  __syncthreads();
}

// (lo, hi) += round(d / 2^u) in 128-bit two's complement, integer operations
// only; zero and subnormal d add nothing (far below any unit used here), a
// non-finite d or one beyond the 128-bit range sets bad.
__device__ __forceinline__ void add_fixed128(unsigned long long& lo, unsigned long long& hi, double d, int u,
                                             bool& bad) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return;
  if (ex == 0x7FF) {
    bad = true;
    return;
  }
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const int sh = (ex - 1075) - u;
  if (sh > 72) {
    bad = true;
    return;
  }
  add_shifted128(lo, hi, (b >> 63) ? -m : m, sh);
}

// End of k_spmv_dots: in the last CTA, the column finish and, from the exact
// fixed-point dot sums, the MGS coefficients H(i, j) (Algorithm 1, inner
// loop).  buf: blockDim.x doubles.
template <typename T, int NW, bool SK>
__device__ __forceinline__ void spmv_dots_finish(const WS& ws, const Win<T>& win, int j, int grid2, const int* du,
                                                 double* buf, unsigned long long* redu) {
  Ctl* c = ws.ctl;
  if (last_block(&c->counter)) {
    if (j >= 1) finish_column(ws, j, grid2, buf, redu);
    unsigned long long wmv = 0ull;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
      const unsigned long long u =
          (unsigned long long)__double_as_longlong(__ldcg(ws.part + (int64_t)b * NPART + T_MAX));
      wmv = u > wmv ? u : wmv;
    }
    const unsigned long long wmx = block_max_u64(wmv, redu);
    const bool finite = bexp_of_bits(wmx) != 0x7FF;
    double p[NW];
#pragma unroll
    for (int a = 0; a < NW; ++a) {
      const unsigned long long* acc = ws.dacc + ((int64_t)j * T_MAX + a) * 2;
      p[a] = finite ? i128_to_double(__ldcg(acc), __ldcg(acc + 1), du[a]) : __longlong_as_double(0x7FF8000000000000ll);
    }
    if (threadIdx.x == 0) {
      // Truncated MGS (Algorithm 1, inner loop) from the dots: with
      // v_i = alpha_i v_hat_i and w_true = alpha_j w,
      // H(i,j) = v_i . (w_true - sum_{l<i} H(l,j) v_l).
      const int t = ws.t;
      const double aj = c->alpha[j];
      double h[NW];
      double bound = fabs(aj) * __longlong_as_double((long long)wmx);
      c->coef[0] = aj;
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        const int i = win.lo + a;
        const double ai = c->alpha[i];
        double v = ai * aj * p[a];
#pragma unroll
        for (int b2 = 0; b2 < a; ++b2) {
          const int l = win.lo + b2;
          v -= h[b2] * ai * c->alpha[l] * c->gram[i][i - l - 1];
        }
        h[a] = v;
        c->hband[j][i - j + t - 1] = v;
        c->coef[1 + a] = v * ai;
        bound += fabs(c->coef[1 + a]) * __longlong_as_double((long long)c->vmax[i]);
      }
      c->wmax = wmx;
      c->vtop[j + 1] = window_top(bound * (1.0 + 1e-12), ws.win_bits);
      atomicAdd(&c->matvecs, 1);
      if (SK) atomicAdd(&c->sketches, 1);
    }
  }
}

// ---------------------------------------------------------------------------
// Arnoldi step j, part 1: w = A v_hat_j (one thread per row) with the dots of
// w against the truncation window, and, for j >= 1, the sketch S v_hat_j of
// the vector being multiplied (tile by tile, on the integer and load/store
// pipes while the FP64 pipe runs the SpMV).  The last CTA finishes column j
// and turns the dots into the MGS coefficients H(i, j).
// ---------------------------------------------------------------------------
template <typename T, int NW, bool SK, int RPT>  // NW window vectors v_hat_lo .. v_hat_j; SK: sketch v_hat_j;
                                                 // RPT sketch rows per thread (s <= RPT SK_THREADS)
__global__ void __launch_bounds__(SK_THREADS, 3) k_spmv_dots(WS ws, CsrDev A, Win<T> win, int j, int grid2) {
  Ctl* c = ws.ctl;
  if (arnoldi_stopped(c, j)) return;
  extern __shared__ unsigned char smem[];
  const int tileR = sketch_tile_rows(ws.zeta);
  double* vals = (double*)smem;
  uint16_t* ent_s = (uint16_t*)(vals + tileR);
  uint16_t* ptr_s = ent_s + tileR * ws.zeta;
  __shared__ double buf[SK_THREADS];
  __shared__ unsigned long long redu[32];
  // per-thread window-dot accumulators, fixed point (see add_fixed128)
  __shared__ unsigned long long dlo[NW][SK_THREADS], dhi[NW][SK_THREADS];
  const T* __restrict__ x = win.v[NW - 1];
  T* __restrict__ w = (T*)ws.Wv;
  const int top = SK ? c->vtop[j] : 0;
  T d[NW];
#pragma unroll
  for (int a = 0; a < NW; ++a) d[a] = 0;
  unsigned long long wm = 0ull;
  unsigned long long lo[RPT], hi[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) lo[k] = hi[k] = 0ull;
  const int64_t n = A.n;
  const int ntiles = (int)((n + tileR - 1) / tileR);
  // Fixed-point units of the window dots: |w_r| <= ||A||_inf max|v_hat_j| and
  // |v_hat_i,r| <= max|v_hat_i|, so |dot_a| < 2^E with E from the exponents of
  // n, ||A||_inf and the two maxima; the unit 2^(E - 120) keeps every sum
  // within 128 bits and 2^-120 of the bound (max|v_hat_j| is bounded by the
  // window top the previous step set; for j = 0 it is max|r0|).
  int du[NW];
  bool dbad = false;
  {
    const int ex = j == 0 ? bexp_of_bits(c->vmax[0]) - 1022 : c->vtop[j] - ws.win_bits - 2;
    const int ea = bexp_of_bits((unsigned long long)__double_as_longlong(c->anorm_inf)) - 1022;
    const int en = 64 - __clzll((long long)n);
#pragma unroll
    for (int a = 0; a < NW; ++a) {
      const int i = win.lo + a;
      const int ev = i == j ? ex : bexp_of_bits(c->vmax[i]) - 1022;
      du[a] = en + ea + ex + ev - 120;
      dlo[a][threadIdx.x] = 0ull;
      dhi[a][threadIdx.x] = 0ull;
    }
  }
  // Tiles are handed out by a counter, so CTAs that start late (an SM shared
  // with the dense step on the other stream) take fewer tiles.
  __shared__ int next_tile;
  int* __restrict__ tctr = ws.tctr + j;
  if (threadIdx.x == 0) next_tile = atomicAdd(tctr, 1);
  __syncthreads();
  for (int tile = next_tile; tile < ntiles; tile = next_tile) {
    __syncthreads();  // every thread holds this tile's index before it is replaced
    // the next tile's claim is published at the end of this one (its latency
    // hides behind the tile's work)
    int claimed = 0;
    if (threadIdx.x == 0) claimed = atomicAdd(tctr, 1);
    const int64_t r0 = (int64_t)tile * tileR;
    const int ncols = (int)(n - r0 < (int64_t)tileR ? n - r0 : (int64_t)tileR);
    if (SK) tile_sketch_prefetch(ws, tileR, tile, ent_s, ptr_s);
    // two rows per thread at a time (i and i + blockDim.x), so that each
    // thread has both rows' loads in flight
    for (int i = threadIdx.x; i < tileR; i += 2 * blockDim.x) {
      const int ib = i + blockDim.x;
      const bool va_ = i < ncols, vb_ = ib < ncols;
      const int64_t ra = r0 + i, rb = r0 + ib;
      T wa[NW], wb[NW];
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        wa[a] = va_ ? win.v[a][ra] : (T)0;
        wb[a] = vb_ ? win.v[a][rb] : (T)0;
      }
      T ya = 0, yb = 0;
      csr_row_pair<T>(A, x, ra, va_, rb, vb_, ya, yb);
      if (va_) {
        w[ra] = ya;
#pragma unroll
        for (int a = 0; a < NW; ++a) d[a] = fma(wa[a], ya, d[a]);
        const unsigned long long u = abs_bits((double)ya);
        wm = u > wm ? u : wm;
      }
      if (vb_) {
        w[rb] = yb;
#pragma unroll
        for (int a = 0; a < NW; ++a) d[a] = fma(wb[a], yb, d[a]);
        const unsigned long long u = abs_bits((double)yb);
        wm = u > wm ? u : wm;
      }
      if (SK) {
        vals[i] = va_ ? (double)x[ra] : 0.0;
        if (ib < tileR) vals[ib] = vb_ ? (double)x[rb] : 0.0;
      }
    }
    if (SK) tile_sketch_accumulate<RPT>(ws, ncols, vals, ent_s, ptr_s, redu, top, lo, hi);
    // this thread's rows of the tile, summed in order, join its exact
    // fixed-point accumulators: the dots then do not depend on which CTA took
    // which tile
#pragma unroll
    for (int a = 0; a < NW; ++a) {
      add_fixed128(dlo[a][threadIdx.x], dhi[a][threadIdx.x], (double)d[a], du[a], dbad);
      d[a] = 0;
    }
    if (threadIdx.x == 0) next_tile = claimed;
    __syncthreads();  // next_tile is published
  }
  if (SK) {
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int row = threadIdx.x + k * blockDim.x;
      if (row < ws.s) atomic_add128(ws.accV + (int64_t)j * 2 * S_MAX + 2 * row, lo[k], hi[k]);
    }
  }
  // the CTA's dot sums (exact), its max |w| (non-finite when a partial was)
  for (int st = SK_THREADS / 2; st > 0; st >>= 1) {
    __syncthreads();
    if ((int)threadIdx.x < st) {
#pragma unroll
      for (int a = 0; a < NW; ++a) {
        const unsigned long long l0 = dlo[a][threadIdx.x], l1 = dlo[a][threadIdx.x + st];
        const unsigned long long nl = l0 + l1;
        dhi[a][threadIdx.x] += dhi[a][threadIdx.x + st] + (nl < l0 ? 1ull : 0ull);
        dlo[a][threadIdx.x] = nl;
      }
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < NW) atomic_add128(ws.dacc + ((int64_t)j * T_MAX + threadIdx.x) * 2,
                                           dlo[threadIdx.x][0], dhi[threadIdx.x][0]);
  if (dbad) wm = 0x7FF8000000000000ull;
  wm = block_max_u64(wm, redu);
  if (threadIdx.x == 0) ws.part[blockIdx.x * NPART + T_MAX] = __longlong_as_double((long long)wm);
  spmv_dots_finish<T, NW, SK>(ws, win, j, grid2, du, buf, redu);
}

int update_grid(const WS& ws) {
  const int g = (ws.grid_max / 8) * 3;  // three CTAs per SM, many rows per thread (two and four ran slower)
  return g < 1 ? 1 : g;
}

template <typename T, int NW, bool SK>
static cudaError_t launch_spmv_t(const WS& ws, CsrDev A, const Win<T>& win, int j, cudaStream_t st) {
  // the instance with two sketch rows per thread for s <= 512 (the common case; fewer
  // registers), three otherwise
  const bool wide = SK && ws.s > SK_RPT_SMALL * SK_THREADS;
  static bool attr = false, attr_w = false;
  cudaError_t e = wide ? set_smem((const void*)k_spmv_dots<T, NW, SK, SK_RPT>, sketch_smem_bytes(ZETA_MAX), attr_w)
                       : set_smem((const void*)k_spmv_dots<T, NW, SK, SK_RPT_SMALL>, sketch_smem_bytes(ZETA_MAX), attr);
  if (e != cudaSuccess) return e;
  const size_t sm = SK ? sketch_smem_bytes(ws.zeta) : 0;
  // three CTAs per SM are resident (register budget); tiles are handed out by a counter
  int g = grid_tiles(ws, A.n);
  const int g3 = 3 * (ws.grid_max / 8);
  if (g > g3) g = g3;
  if (wide)
    k_spmv_dots<T, NW, SK, SK_RPT><<<g, SK_THREADS, sm, st>>>(ws, A, win, j, update_grid(ws));
  else
    k_spmv_dots<T, NW, SK, SK_RPT_SMALL><<<g, SK_THREADS, sm, st>>>(ws, A, win, j, update_grid(ws));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmv_dots(const WS& ws, CsrDev A, const T* const* vcol, int j, cudaStream_t st) {
  Win<T> win;
  win.lo = j - ws.t + 1 > 0 ? j - ws.t + 1 : 0;
  win.nw = j - win.lo + 1;
  for (int a = 0; a < T_MAX; ++a) win.v[a] = a < win.nw ? vcol[win.lo + a] : nullptr;
  if (j == 0) return launch_spmv_t<T, 1, false>(ws, A, win, j, st);  // S r0 came with r0
  if (ws.sketch_kind) {  // the DCT sketch of v_hat_j is a separate launch before this one
    switch (win.nw) {
      case 1: return launch_spmv_t<T, 1, false>(ws, A, win, j, st);
      case 2: return launch_spmv_t<T, 2, false>(ws, A, win, j, st);
      case 3: return launch_spmv_t<T, 3, false>(ws, A, win, j, st);
      default: return launch_spmv_t<T, 4, false>(ws, A, win, j, st);
    }
  }
  switch (win.nw) {
    case 1: return launch_spmv_t<T, 1, true>(ws, A, win, j, st);
    case 2: return launch_spmv_t<T, 2, true>(ws, A, win, j, st);
    case 3: return launch_spmv_t<T, 3, true>(ws, A, win, j, st);
    default: return launch_spmv_t<T, 4, true>(ws, A, win, j, st);
  }
}

// S v_hat_j for the last column of a cycle (no SpMV follows it), with the
// column's finish.
template <typename T>
__global__ void __launch_bounds__(SK_THREADS) k_sketch_col(WS ws, const T* __restrict__ x, int j, int grid2) {
  Ctl* c = ws.ctl;
  if (arnoldi_stopped(c, j)) return;
  extern __shared__ unsigned char smem[];
  const int tileR = sketch_tile_rows(ws.zeta);
  double* vals = (double*)smem;
  uint16_t* ent_s = (uint16_t*)(vals + tileR);
  uint16_t* ptr_s = ent_s + tileR * ws.zeta;
  __shared__ double buf[SK_THREADS];
  __shared__ unsigned long long redu[32];
  const int top = c->vtop[j];
  unsigned long long lo[SK_RPT], hi[SK_RPT];
#pragma unroll
  for (int k = 0; k < SK_RPT; ++k) lo[k] = hi[k] = 0ull;
  const int64_t n = ws.n;
  const int ntiles = (int)((n + tileR - 1) / tileR);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * tileR;
    const int ncols = (int)(n - r0 < (int64_t)tileR ? n - r0 : (int64_t)tileR);
    if (!ws.sketch_kind) tile_sketch_prefetch(ws, tileR, tile, ent_s, ptr_s);
    for (int i = threadIdx.x; i < tileR; i += blockDim.x) vals[i] = i < ncols ? (double)x[r0 + i] : 0.0;
    if (ws.sketch_kind)
      tile_dct_accumulate<SK_RPT>(ws, r0, ncols, vals, top, lo, hi);
    else
      tile_sketch_accumulate<SK_RPT>(ws, ncols, vals, ent_s, ptr_s, redu, top, lo, hi);
  }
#pragma unroll
  for (int k = 0; k < SK_RPT; ++k) {
    const int row = threadIdx.x + k * blockDim.x;
    if (row < ws.s) atomic_add128(ws.accV + (int64_t)j * 2 * S_MAX + 2 * row, lo[k], hi[k]);
  }
  if (last_block(&c->counter)) {
    finish_column(ws, j, grid2, buf, redu);
    if (threadIdx.x == 0) atomicAdd(&c->sketches, 1);
  }
}

template <typename T>
cudaError_t launch_sketch_col(const WS& ws, const T* x, int j, cudaStream_t st) {
  static bool attr = false;
  cudaError_t e = set_smem((const void*)k_sketch_col<T>, sketch_smem_bytes(ZETA_MAX), attr);
  if (e != cudaSuccess) return e;
  k_sketch_col<T><<<grid_tiles(ws, ws.n), SK_THREADS, sketch_smem_bytes(ws.zeta), st>>>(ws, x, j, update_grid(ws));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Arnoldi step j, part 2: v_hat_{j+1} = a_0 w - sum_i a_i v_hat_i, with
// ||v_hat_{j+1}||^2, its dots with the t-1 newest window vectors and its max
// magnitude as per-CTA partials (part2).  Pure streaming: many rows per thread.
// In FP64 the update itself takes three FP64 operations per row; the squared
// norm and the window dots run on the integer pipe instead (eidot.cuh): each
// row's v_hat_{j+1} is rounded to 52 bits of the bound the SpMV recorded for
// it (|v_hat_{j+1}| < 2^E, E = vtop[j+1] - win_bits - 2), each window entry to
// 52 bits of its column's maximum, and the products are summed exactly; the
// thread's sums are rounded to FP64 once every UPD_FLUSH rows.  A non-finite
// v_hat_{j+1} makes the CTA's norm partial NaN (the column is then a breakdown).
// ---------------------------------------------------------------------------
constexpr int UPD_FLUSH = 1024;  // rows per exact integer run (Acc3 holds 2048 terms)

// q52 for a value that may break the vector's bound (a non-finite one): 0 then;
// the caller flags non-finite values through the maximum.
__device__ __forceinline__ Q52 q52_safe(double x, int emax) {
  const int ex = bexp(x);
  if (ex > emax) return Q52{0, 0u};
  return q52(x, emax, 0);
}

template <typename T, int NW, int NC>  // NW window vectors, NC = t - 1 dots kept for the next window
__global__ void __launch_bounds__(256) k_update(WS ws, Win<T> win, T* __restrict__ vnext, int j) {
  Ctl* c = ws.ctl;
  if (arnoldi_stopped(c, j)) return;
  __shared__ double buf[256];
  __shared__ unsigned long long redu[32];
  constexpr bool kExact = std::is_same<T, double>::value;
  T cf[NW + 1];
#pragma unroll
  for (int a = 0; a <= NW; ++a) cf[a] = (T)c->coef[a];
  const T* __restrict__ w = (const T*)ws.Wv;
  constexpr int NCX = NC > 0 ? NC : 1;
  double nrm_d = 0.0, cr_d[NCX];
  T nrm = 0;
  T cr[NCX];
#pragma unroll
  for (int q = 0; q < NCX; ++q) {
    cr[q] = 0;
    cr_d[q] = 0.0;
  }
  // fixed-point exponents (biased): v_hat_{j+1} against its bound, window columns
  // against their maxima
  const int ev = c->vtop[j + 1] - ws.win_bits - 2 + 1022;
  int ew[NCX];
#pragma unroll
  for (int q = 0; q < NCX; ++q) ew[q] = (q < NC && q < NW) ? bexp_of_bits(c->vmax[win.lo + NW - 1 - q]) : 0;
  Acc3 an, ac[NCX];
  an.zero();
#pragma unroll
  for (int q = 0; q < NCX; ++q) ac[q].zero();
  int run = 0;
  unsigned long long vm = 0ull;
  const int64_t n = ws.n, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
    T wv[NW];
#pragma unroll
    for (int a = 0; a < NW; ++a) wv[a] = win.v[a][r];
    T v = cf[0] * w[r];
#pragma unroll
    for (int a = 0; a < NW; ++a) v = fma(-cf[1 + a], wv[a], v);
    vnext[r] = v;
    if constexpr (kExact) {
      const Q52 qv = q52_safe((double)v, ev);
      an.mac(qv, qv);
#pragma unroll
      for (int q = 0; q < NC; ++q)
        if (q < NW) ac[q].mac(qv, q52_safe((double)wv[NW - 1 - q], ew[q]));
      if (++run == UPD_FLUSH) {
        nrm_d += acc_to_double(an, 2 * (ev - 1073));
        an.zero();
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          cr_d[q] += acc_to_double(ac[q], (ev - 1073) + (ew[q] - 1073));
          ac[q].zero();
        }
        run = 0;
      }
    } else {
      nrm = fma(v, v, nrm);
#pragma unroll
      for (int q = 0; q < NC; ++q)
        if (q < NW) cr[q] = fma(v, wv[NW - 1 - q], cr[q]);
    }
    const unsigned long long u = abs_bits((double)v);
    vm = u > vm ? u : vm;
  }
  if constexpr (kExact) {
    nrm_d += acc_to_double(an, 2 * (ev - 1073));
#pragma unroll
    for (int q = 0; q < NC; ++q) cr_d[q] += acc_to_double(ac[q], (ev - 1073) + (ew[q] - 1073));
  } else {
    nrm_d = (double)nrm;
#pragma unroll
    for (int q = 0; q < NC; ++q) cr_d[q] = (double)cr[q];
  }
  const double nrm_b = block_sum_lean(nrm_d, buf);
  double cr_b[NCX];
#pragma unroll
  for (int q = 0; q < NC; ++q) cr_b[q] = block_sum_lean(cr_d[q], buf);
  vm = block_max_u64(vm, redu);
  if (threadIdx.x == 0) {
    double* pp = ws.part2 + blockIdx.x * NPART;
    // a non-finite entry (its magnitude bits at or above those of Inf) poisons the norm
    pp[0] = vm >= 0x7FF0000000000000ull ? __longlong_as_double(0x7FF8000000000000ll) : nrm_b;
#pragma unroll
    for (int q = 0; q < NC; ++q) pp[1 + q] = cr_b[q];
    pp[T_MAX] = __longlong_as_double((long long)vm);
  }
}

template <typename T, int NW, int NC>
static cudaError_t launch_upd(const WS& ws, const Win<T>& win, T* vnext, int j, cudaStream_t st) {
  k_update<T, NW, NC><<<update_grid(ws), 256, 0, st>>>(ws, win, vnext, j);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_sketch(const WS& ws, const T* const* vcol, T* vnext, int j, cudaStream_t st) {
  Win<T> win;
  win.lo = j - ws.t + 1 > 0 ? j - ws.t + 1 : 0;
  win.nw = j - win.lo + 1;
  for (int a = 0; a < T_MAX; ++a) win.v[a] = a < win.nw ? vcol[win.lo + a] : nullptr;
  const int nc = ws.t - 1;
  switch (win.nw * 10 + nc) {
    case 10: return launch_upd<T, 1, 0>(ws, win, vnext, j, st);
    case 11: return launch_upd<T, 1, 1>(ws, win, vnext, j, st);
    case 12: return launch_upd<T, 1, 2>(ws, win, vnext, j, st);
    case 13: return launch_upd<T, 1, 3>(ws, win, vnext, j, st);
    case 21: return launch_upd<T, 2, 1>(ws, win, vnext, j, st);
    case 22: return launch_upd<T, 2, 2>(ws, win, vnext, j, st);
    case 23: return launch_upd<T, 2, 3>(ws, win, vnext, j, st);
    case 32: return launch_upd<T, 3, 2>(ws, win, vnext, j, st);
    case 33: return launch_upd<T, 3, 3>(ws, win, vnext, j, st);
    case 43: return launch_upd<T, 4, 3>(ws, win, vnext, j, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Tall products with [U, V] on the integer pipe (see eidot.cuh).  Column l of
// W = [U, V(:, 0:j)] is scaled by 2^delta_l so that its largest magnitude lies
// in [0.5, 1); all elements then share one fixed-point unit 2^-51, and the
// coefficients carry the inverse scales (prepared by the dense kernels).
// ---------------------------------------------------------------------------
template <typename T>
struct Cols {
  const T* v0;  // column 0 of V (the cycle's residual)
  const T* vs;  // columns 1.. (column c at vs + (c-1)*ldv)
};

template <typename T>
__device__ __forceinline__ const T* wcol(const T* U, const Cols<T>& V, int64_t ld, int kh, int l) {
  return l < kh ? U + (int64_t)l * ld : (l == kh ? V.v0 : V.vs + (int64_t)(l - kh - 1) * ld);
}

// delta_l = -(frexp exponent of the column's max |.|), from recorded maxima.
__device__ __forceinline__ int col_delta(const Ctl* c, int ubuf, int kh, int l) {
  const unsigned long long mb = l < kh ? c->umax[ubuf][l] : c->vmax[l - kh];
  const int e = bexp_of_bits(mb);
  return e == 0 ? 0 : -(e - 1022);
}

// x_trial = x + W y'  (one thread per row).
template <typename T>
__global__ void __launch_bounds__(256) k_check_q(WS ws, const T* __restrict__ U, Cols<T> V,
                                                 const T* __restrict__ xcur, T* __restrict__ xtrial,
                                                 int kh, int j, int ubuf) {
  Ctl* c = ws.ctl;
  if (!c->check) return;
  __shared__ Q52 yq[D_MAX];
  __shared__ int dl[D_MAX];
  __shared__ unsigned long long redu[32];
  const int d = kh + j + 1;
  for (int l = threadIdx.x; l < d; l += blockDim.x) {
    const unsigned long long b = ws.ytq[l];
    yq[l].hi = (int)(b >> 32);
    yq[l].lo = (unsigned)(b & 0xFFFFFFFFull);
    dl[l] = col_delta(c, ubuf, kh, l);
  }
  __syncthreads();
  const int sexp = (1022 - 1022) - 51 + ws.yexp[0] - 51;
  const int64_t ld = ws.ldv;
  unsigned long long xm = 0ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ws.n; r += (int64_t)gridDim.x * blockDim.x) {
    Acc3 acc;
    acc.zero();
    int l = 0;
    for (; l + 4 <= d; l += 4) {
      const double w0 = (double)wcol(U, V, ld, kh, l)[r], w1 = (double)wcol(U, V, ld, kh, l + 1)[r];
      const double w2 = (double)wcol(U, V, ld, kh, l + 2)[r], w3 = (double)wcol(U, V, ld, kh, l + 3)[r];
      acc.mac(q52(w0, 1022, dl[l]), yq[l]);
      acc.mac(q52(w1, 1022, dl[l + 1]), yq[l + 1]);
      acc.mac(q52(w2, 1022, dl[l + 2]), yq[l + 2]);
      acc.mac(q52(w3, 1022, dl[l + 3]), yq[l + 3]);
    }
    for (; l < d; ++l) acc.mac(q52((double)wcol(U, V, ld, kh, l)[r], 1022, dl[l]), yq[l]);
    const T v = (T)((double)xcur[r] + acc_to_double(acc, sexp));
    xtrial[r] = v;
    const unsigned long long u = abs_bits((double)v);
    xm = u > xm ? u : xm;
  }
  xm = block_max_u64(xm, redu);
  if (threadIdx.x == 0) atomicMax(&c->xmax, xm);
}

template <typename T>
cudaError_t launch_check_gemv(const WS& ws, const T* U, const T* const* vcol, const T* xcur,
                              T* xtrial, int kh, int j, int ubuf, cudaStream_t st) {
  Cols<T> V{vcol[0], (const T*)ws.Vs};
  k_check_q<T><<<grid_rows(ws.n, 256, ws.grid_max), 256, 0, st>>>(ws, U, V, xcur, xtrial, kh, j, ubuf);
  return cudaGetLastError();
}

// U_new = W P' for W wider than the shared-memory tile of k_recycle_rb.  A CTA stages RT rows of W as
// fixed-point values in shared memory; thread (r, g) accumulates row r against
// columns 8g .. 8g+7 of P'' (read through L1: every lane of a warp reads the
// same coefficient).
constexpr int RT = 32;
template <typename T>
__global__ void __launch_bounds__(128, 4) k_recycle_q(WS ws, const T* __restrict__ U, Cols<T> V,
                                                      T* __restrict__ Unew, int kh, int ucur, int unext) {
  Ctl* c = ws.ctl;
  const int kp = c->kprime, jf = c->jf;
  if (kp <= 0 || jf <= 0) return;
  const int d = kh + jf;
  extern __shared__ unsigned long long smq[];
  Q52* tile = (Q52*)smq;  // [d][RT]
  __shared__ int dl[D_MAX];
  __shared__ int fx[K_MAX];
  for (int l = threadIdx.x; l < d; l += blockDim.x) dl[l] = col_delta(c, ucur, kh, l);
  for (int cc = threadIdx.x; cc < K_MAX; cc += blockDim.x) fx[cc] = ws.Pexp[cc];
  __syncthreads();
  const int64_t ld = ws.ldv, n = ws.n;
  const int r = threadIdx.x % RT, g = threadIdx.x / RT;
  const int ngroups = (kp + 7) / 8;
  unsigned long long um[8] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  const int64_t ntiles = (n + RT - 1) / RT;
  const int step = blockDim.x / RT;
  for (int64_t tile_i = blockIdx.x; tile_i < ntiles; tile_i += gridDim.x) {
    const int64_t r0 = tile_i * RT;
    const int nr = (int)(n - r0 < RT ? n - r0 : RT);
    for (int l0 = g; l0 < d; l0 += 8 * step) {  // issue eight loads before converting any
      double w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int l = l0 + u * step;
        w[u] = (l < d && r < nr) ? (double)wcol(U, V, ld, kh, l)[r0 + r] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int l = l0 + u * step;
        if (l < d) tile[l * RT + r] = q52(w[u], 1022, dl[l]);
      }
    }
    __syncthreads();
    for (int gg = g; gg < ngroups; gg += step) {
      Acc3 acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q].zero();
      const unsigned long long* __restrict__ yc = ws.Pq + (int64_t)(gg * 8) * D_MAX;
      for (int l = 0; l < d; ++l) {
        const Q52 x = tile[l * RT + r];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const unsigned long long yb = __ldg(yc + q * D_MAX + l);  // packed (hi << 32) | lo
          Q52 y;
          y.hi = (int)(yb >> 32);
          y.lo = (unsigned)(yb & 0xFFFFFFFFull);
          acc[q].mac(x, y);
        }
      }
      if (r < nr) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = gg * 8 + q;
          if (col < kp) {
            const T v = (T)acc_to_double(acc[q], -51 + fx[col] - 51);
            Unew[r0 + r + (int64_t)col * ld] = v;
            const unsigned long long u = abs_bits((double)v);
            if (gg == g) um[q] = u > um[q] ? u : um[q];
            else atomicMax(&c->umax[unext][col], u);
          }
        }
      }
    }
    __syncthreads();
  }
  if (g < ngroups) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int col = g * 8 + q;
      unsigned long long u = warp_max_u64(um[q]);
      if ((threadIdx.x & 31) == 0 && col < kp && u) atomicMax(&c->umax[unext][col], u);
    }
  }
}

// U_new = W P' for the kprime recycle columns (W = [U, V(:, 0:jf)]), as an
// exact integer product on the 32-bit multiply-add pipe.  Two CTAs share an
// SM (one stages its tile while the other multiplies) and walk over tiles of
// RB_ROWS rows: the tile of W is quantised into shared memory once (column l
// scaled by 2^delta_l, unit 2^-51), and warp w computes columns
// w*CPT .. w*CPT+CPT-1 of the tile, lane i the rows i and i+32.  Each product X Y of 52-bit integers
// X = xh 2^26 + xl, Y = yh 2^26 + yl takes three 32x32->64 multiply-adds
// (Karatsuba): xh yh, xl yl and (xh + xl)(yh + yl); the cross term is their
// difference.  Every sum is exact (|terms| < 2^54, at most D_MAX of them), so
// the result equals the exactly rounded product of the quantised operands.
constexpr int RB_ROWS = 64;
constexpr int RB_RPL = RB_ROWS / 32;  // rows per lane
constexpr int RB_THREADS = 256;

struct __align__(16) YK {
  int hi, lo, sum, pad;
};

template <typename T, int CPT>
__global__ void __launch_bounds__(RB_THREADS, 2) k_recycle_rb(WS ws, const T* __restrict__ U, Cols<T> V,
                                                               T* __restrict__ Unew, int kh, int ucur, int unext,
                                                               int dcap) {
  Ctl* c = ws.ctl;
  const int kp = c->kprime, jf = c->jf;
  if (kp <= 0 || jf <= 0) return;
  const int d = kh + jf;
  constexpr int NCOL = 8 * CPT;
  if (d > dcap || kp > NCOL) {  // cannot happen (d <= kh + m, kp <= k + 1): refuse rather than overrun
    if (threadIdx.x == 0 && blockIdx.x == 0) c->rankfail = 1;
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  YK* ytab = (YK*)smraw;                                      // [dcap][NCOL]
  // [dcap][RB_ROWS]: row r of column l at l*RB_ROWS + 2*(r % 32) + r / 32, so a
  // lane's two rows (r and r + 32) are one 16-byte load
  Q52* xq = (Q52*)(smraw + (size_t)dcap * NCOL * sizeof(YK));
  __shared__ int dl[D_MAX];
  __shared__ int fx[NCOL];
  __shared__ const T* colp[D_MAX];
  for (int l = threadIdx.x; l < d; l += blockDim.x) {
    dl[l] = col_delta(c, ucur, kh, l);
    colp[l] = wcol(U, V, ws.ldv, kh, l);
  }
  for (int q = threadIdx.x; q < NCOL; q += blockDim.x) fx[q] = q < kp ? ws.Pexp[q] : 0;
  for (int idx = threadIdx.x; idx < d * NCOL; idx += blockDim.x) {
    const int l = idx / NCOL, q = idx % NCOL;
    YK y{0, 0, 0, 0};
    if (q < kp) {
      const unsigned long long b = ws.Pq[l + (int64_t)q * D_MAX];  // packed (hi << 32) | lo
      y.hi = (int)(b >> 32);
      y.lo = (int)(unsigned)(b & 0xFFFFFFFFull);
      y.sum = y.hi + y.lo;
    }
    ytab[idx] = y;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t ld = ws.ldv, n = ws.n;
  const int64_t ntiles = (n + RB_ROWS - 1) / RB_ROWS;
  unsigned long long um[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) um[q] = 0ull;
  const bool active = w * CPT < kp;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * RB_ROWS;
    const int nr = (int)(n - r0 < RB_ROWS ? n - r0 : RB_ROWS);
    // stage the tile: eight loads in flight per thread before any is converted
    for (int base = threadIdx.x; base < d * RB_ROWS; base += 8 * RB_THREADS) {
      double wv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * RB_THREADS;
        const int l = idx / RB_ROWS, r = idx % RB_ROWS;
        wv[u] = (idx < d * RB_ROWS && r < nr) ? (double)colp[l][r0 + r] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * RB_THREADS;
        const int l = idx / RB_ROWS, r = idx % RB_ROWS;
        if (idx < d * RB_ROWS) xq[l * RB_ROWS + 2 * (r & 31) + (r >> 5)] = q52(wv[u], 1022, dl[l]);
      }
    }
    __syncthreads();
    if (active) {
      long long hh[RB_RPL][CPT], mm[RB_RPL][CPT];
      unsigned long long ll[RB_RPL][CPT];
#pragma unroll
      for (int i = 0; i < RB_RPL; ++i)
#pragma unroll
        for (int q = 0; q < CPT; ++q) hh[i][q] = mm[i][q] = 0, ll[i][q] = 0ull;
      const YK* yrow = ytab + w * CPT;
      const int4* xrow = (const int4*)(xq + 2 * lane);
      static_assert(RB_RPL == 2, "two rows per lane: one 16-byte load");
#pragma unroll 4
      for (int l = 0; l < d; ++l) {
        const int4 xx = xrow[l * (RB_ROWS / 2)];
        Q52 x[RB_RPL];
        x[0].hi = xx.x;
        x[0].lo = (unsigned)xx.y;
        x[1].hi = xx.z;
        x[1].lo = (unsigned)xx.w;
        int xs[RB_RPL];
#pragma unroll
        for (int i = 0; i < RB_RPL; ++i) xs[i] = x[i].hi + (int)x[i].lo;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const YK y = yrow[l * NCOL + q];
#pragma unroll
          for (int i = 0; i < RB_RPL; ++i) {
            asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(hh[i][q]) : "r"(x[i].hi), "r"(y.hi));
            asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(ll[i][q]) : "r"(x[i].lo), "r"(y.lo));
            asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(mm[i][q]) : "r"(xs[i]), "r"(y.sum));
          }
        }
      }
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        const int col = w * CPT + q;
        if (col >= kp) continue;
#pragma unroll
        for (int i = 0; i < RB_RPL; ++i) {
          const int r = lane + 32 * i;
          if (r >= nr) continue;
          const long long mid = mm[i][q] - hh[i][q] - (long long)ll[i][q];
          unsigned long long lo = ll[i][q], hi = 0ull;
          add_shifted128(lo, hi, mid, 26);
          add_shifted128(lo, hi, hh[i][q], 52);
          const T v = (T)i128_to_double(lo, hi, -51 + fx[col] - 51);
          Unew[r0 + r + (int64_t)col * ld] = v;
          const unsigned long long u = abs_bits((double)v);
          um[q] = u > um[q] ? u : um[q];
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int col = w * CPT + q;
    const unsigned long long u = warp_max_u64(um[q]);
    if (lane == 0 && col < kp && u) atomicMax(&c->umax[unext][col], u);
  }
}

// Shared memory of k_recycle_rb for dcap columns of W and NCOL of P.
static size_t recycle_rb_smem(int dcap, int ncol) {
  return (size_t)dcap * ncol * sizeof(YK) + (size_t)dcap * RB_ROWS * sizeof(Q52);
}
constexpr size_t RB_SMEM_MAX = 112 * 1024;  // two CTAs per SM

template <typename T>
cudaError_t launch_recycle_gemm(const WS& ws, const T* U, const T* const* vcol, T* Unew, int kh,
                                int ucur, int unext, cudaStream_t st) {
  Cols<T> V{vcol[0], (const T*)ws.Vs};
  if (sizeof(T) == sizeof(double) && !ws.recycle_int)
    return launch_recycle_tc(ws, (const double*)U, (const double*)vcol[0], (const double*)ws.Vs, (double*)Unew, kh,
                             ucur, unext, st);
  const int nsm = ws.grid_max / 8;
  const int dcap = kh + ws.m;  // W has kh + jf <= kh + m columns; kprime <= k + 1 = kmax
  const int grid = 2 * nsm;
  if (ws.kmax <= 24 && recycle_rb_smem(dcap, 24) <= RB_SMEM_MAX) {
    const size_t sm = recycle_rb_smem(dcap, 24);
    static bool attr = false;
    cudaError_t e = set_smem((const void*)k_recycle_rb<T, 3>, RB_SMEM_MAX, attr);
    if (e != cudaSuccess) return e;
    k_recycle_rb<T, 3><<<grid, RB_THREADS, sm, st>>>(ws, U, V, Unew, kh, ucur, unext, dcap);
  } else if (recycle_rb_smem(dcap, 32) <= RB_SMEM_MAX) {
    const size_t sm = recycle_rb_smem(dcap, 32);
    static bool attr = false;
    cudaError_t e = set_smem((const void*)k_recycle_rb<T, 4>, RB_SMEM_MAX, attr);
    if (e != cudaSuccess) return e;
    k_recycle_rb<T, 4><<<grid, RB_THREADS, sm, st>>>(ws, U, V, Unew, kh, ucur, unext, dcap);
  } else {
    // wide W (kh + m beyond the shared-memory tile): the row-per-thread kernel
    const size_t sm = (size_t)D_MAX * RT * sizeof(Q52);
    static bool attr = false;
    cudaError_t e = set_smem((const void*)k_recycle_q<T>, sm, attr);
    if (e != cudaSuccess) return e;
    k_recycle_q<T><<<nsm * 4, 128, sm, st>>>(ws, U, V, Unew, kh, ucur, unext);
  }
  return cudaGetLastError();
}

template <typename T>
__global__ void k_spmv(CsrDev A, const T* __restrict__ x, T* __restrict__ y) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.n; r += (int64_t)gridDim.x * blockDim.x)
    y[r] = csr_row_dot<T>(A, x, r);
}

template <typename T>
cudaError_t launch_spmv(CsrDev A, const T* x, T* y, cudaStream_t st) {
  int64_t g = (A.n + 255) / 256;
  if (g > 4096) g = 4096;
  k_spmv<T><<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(A, x, y);
  return cudaGetLastError();
}

// Refined form: the float32 right-hand side of an inner solve, and the float64
// update of the outer iterate.
__global__ void k_to_f32(const double* __restrict__ r64, float* __restrict__ r32, float* __restrict__ d32,
                         int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r32[i] = (float)r64[i];
    d32[i] = 0.f;
  }
}

__global__ void k_add_f32(double* __restrict__ x64, const float* __restrict__ d32, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x64[i] += (double)d32[i];
}

cudaError_t launch_to_f32(const double* r64, float* r32, float* d32, int64_t n, cudaStream_t st) {
  k_to_f32<<<grid_rows(n, 256, 4096), 256, 0, st>>>(r64, r32, d32, n);
  return cudaGetLastError();
}

cudaError_t launch_add_f32(double* x64, const float* d32, int64_t n, cudaStream_t st) {
  k_add_f32<<<grid_rows(n, 256, 4096), 256, 0, st>>>(x64, d32, n);
  return cudaGetLastError();
}

#define SDR_INSTANTIATE_ARNOLDI(T)                                                                          \
  template cudaError_t launch_solve_init_x<T>(const WS&, CsrDev, const T*, const T*, double, cudaStream_t, bool); \
  template cudaError_t launch_residual<T>(const WS&, CsrDev, const T*, const T*, T*, unsigned long long*, int, \
                                          int, cudaStream_t);                                                 \
  template cudaError_t launch_spmv_dots<T>(const WS&, CsrDev, const T* const*, int, cudaStream_t);            \
  template cudaError_t launch_update_sketch<T>(const WS&, const T* const*, T*, int, cudaStream_t);            \
  template cudaError_t launch_check_gemv<T>(const WS&, const T*, const T* const*, const T*, T*, int, int, int, \
                                            cudaStream_t);                                                    \
  template cudaError_t launch_recycle_gemm<T>(const WS&, const T*, const T* const*, T*, int, int, int,        \
                                              cudaStream_t);                                                  \
  template cudaError_t launch_spmv<T>(CsrDev, const T*, T*, cudaStream_t);                                    \
  template cudaError_t launch_sketch_col<T>(const WS&, const T*, int, cudaStream_t);
SDR_INSTANTIATE_ARNOLDI(double)
SDR_INSTANTIATE_ARNOLDI(float)

}  // namespace sdr
