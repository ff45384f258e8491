// Streaming kernels of one GMRES-SDR cycle (Algorithm 1), FP64.
//
//  k_spmv_dots     w = A v_j and the dots of w with the truncation window;
//                  the last CTA turns them into the MGS coefficients H(i, j).
//  k_update_sketch v_hat_{j+1} = w - sum_i H(i,j) v_i (truncated Arnoldi), its
//                  norm and window dots, and S v_hat_{j+1} (one sketch per step).
//  k_residual      r = b - A x with ||r|| and S r; applies the residual control
//                  of Section 3.3 when it serves a true-residual check.
//  k_check_gemv    x_trial = x + [U V] y_tilde.
//  k_recycle_gemm  U_new = [U V] P (recycle update, Section 3.4).
//
// Basis columns are stored unnormalised (v_hat); alpha_c = 1/||v_hat_c|| lives
// in the control block and is folded into every coefficient that touches a
// column, which saves a normalisation pass per step.
#include "launch.cuh"

namespace sdr {

struct Win {
  const double* v[T_MAX];  // v_hat_lo .. v_hat_j
  int lo, nw;
};

__device__ inline double csr_row_dot(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, const double* __restrict__ x, int64_t r) {
  int p0 = rowptr[r], p1 = rowptr[r + 1];
  double y = 0.0;
  for (int p = p0; p < p1; ++p) y = fma(val[p], x[col[p]], y);
  return y;
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
__global__ void k_solve_init(WS ws, CsrDev A, const double* __restrict__ b, const double* __restrict__ x,
                             double rel_tol) {
  __shared__ double red[32];
  __shared__ unsigned long long redu[32];
  double bb = 0.0;
  unsigned long long bm = 0ull, xm = 0ull, am = 0ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.n; r += (int64_t)gridDim.x * blockDim.x) {
    double v = b[r];
    bb = fma(v, v, bb);
    unsigned long long u = abs_bits(v);
    bm = u > bm ? u : bm;
    u = abs_bits(x[r]);
    xm = u > xm ? u : xm;
    double rs = 0.0;
    for (int p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) rs += fabs(A.val[p]);
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
      c->hist_n = 0;
      c->log_n = 0;
      c->matvecs = 0;
      c->sketches = 0;
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

cudaError_t launch_solve_init_x(const WS& ws, CsrDev A, const double* b, const double* x, double rel_tol,
                                cudaStream_t st) {
  k_solve_init<<<grid_rows(A.n, 256, ws.grid_max), 256, 0, st>>>(ws, A, b, x, rel_tol);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// True residual r = b - A x with ||r||, max|r| and S r (tile-fused).
// mode 0: unconditional (solve start).  mode 1: runs only when ctl->check and
// then applies Algorithm 1's residual control in the last CTA.
// ---------------------------------------------------------------------------
__global__ void k_residual(WS ws, CsrDev A, const double* __restrict__ b, const double* __restrict__ x,
                           double* __restrict__ rout, unsigned long long* accR, int j, int mode) {
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
  unsigned long long lo = 0ull, hi = 0ull, rm = 0ull;
  double nrm = 0.0;
  const int64_t n = A.n;
  const int ntiles = (int)((n + tileR - 1) / tileR);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * tileR;
    const int ncols = (int)(n - r0 < (int64_t)tileR ? n - r0 : (int64_t)tileR);
    for (int i = threadIdx.x; i < tileR; i += blockDim.x) {
      double v = 0.0;
      if (i < ncols) {
        int64_t r = r0 + i;
        v = b[r] - csr_row_dot(A.rowptr, A.col, A.val, x, r);
        rout[r] = v;
        nrm = fma(v, v, nrm);
        unsigned long long u = abs_bits(v);
        rm = u > rm ? u : rm;
      }
      vals[i] = v;
    }
    __syncthreads();
    tile_sketch_accumulate(ws, tileR, tile, ncols, vals, ent_s, ptr_s, redu, top, lo, hi);
  }
  if (threadIdx.x < ws.s) atomic_add128(accR + 2 * threadIdx.x, lo, hi);
  nrm = block_sum(nrm, red);
  rm = block_max_u64(rm, redu);
  if (threadIdx.x == 0) {
    ws.part[blockIdx.x * NPART + 0] = nrm;
    ws.part[blockIdx.x * NPART + 1] = __longlong_as_double((long long)rm);
  }
  if (last_block(&c->counter)) {
    double s = reduce_parts(ws.part, gridDim.x, 0, red);
    unsigned long long m = reduce_parts_max(ws.part, gridDim.x, 1, redu);
    if (threadIdx.x == 0) {
      double res = sqrt(s);
      c->res = res;
      c->rmax = m;
      c->accR_top = top;
      c->matvecs += 1;
      c->sketches += 1;
      if (mode == 1) {
        c->nchecks += 1;
        c->check = 0;
        if (res < c->tol) {
          c->converged = 1;
          c->done = 1;
          c->jf = j + 1;
        } else {
          c->safety = c->sres > 0.0 ? res / c->sres : c->safety;  // increase the safety factor
          if (j == ws.m - 1 || c->breakdown) {
            c->done = 1;
            c->jf = j + 1;
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
  int g = ntiles < ws.grid_max ? ntiles : ws.grid_max;
  return g < 1 ? 1 : g;
}

cudaError_t launch_residual(const WS& ws, CsrDev A, const double* b, const double* x, double* rout,
                            unsigned long long* accR, int j, int mode, cudaStream_t st) {
  size_t sm = sketch_smem_bytes(ws.zeta);
  static bool attr = false;
  cudaError_t e = set_smem((const void*)k_residual, sketch_smem_bytes(ZETA_MAX), attr);
  if (e != cudaSuccess) return e;
  k_residual<<<grid_tiles(ws, A.n), 512, sm, st>>>(ws, A, b, x, rout, accR, j, mode);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Arnoldi step j, part 1: w = A v_hat_j, dots with the window, MGS coefficients.
// ---------------------------------------------------------------------------
__global__ void k_spmv_dots(WS ws, CsrDev A, Win win, int j) {
  Ctl* c = ws.ctl;
  if (c->done) return;
  __shared__ double red[32];
  __shared__ unsigned long long redu[32];
  const double* __restrict__ x = win.v[win.nw - 1];
  double* __restrict__ w = ws.Wv;
  double d[T_MAX] = {0.0, 0.0, 0.0, 0.0};
  unsigned long long wm = 0ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.n; r += (int64_t)gridDim.x * blockDim.x) {
    double y = csr_row_dot(A.rowptr, A.col, A.val, x, r);
    w[r] = y;
#pragma unroll
    for (int a = 0; a < T_MAX; ++a)
      if (a < win.nw) d[a] = fma(win.v[a][r], y, d[a]);
    unsigned long long u = abs_bits(y);
    wm = u > wm ? u : wm;
  }
#pragma unroll
  for (int a = 0; a < T_MAX; ++a)
    if (a < win.nw) d[a] = block_sum(d[a], red);
  wm = block_max_u64(wm, redu);
  if (threadIdx.x == 0) {
    double* pp = ws.part + blockIdx.x * NPART;
    for (int a = 0; a < win.nw; ++a) pp[a] = d[a];
    pp[T_MAX] = __longlong_as_double((long long)wm);
  }
  if (last_block(&c->counter)) {
    double p[T_MAX];
#pragma unroll
    for (int a = 0; a < T_MAX; ++a) p[a] = a < win.nw ? reduce_parts(ws.part, gridDim.x, a, red) : 0.0;
    unsigned long long wmx = reduce_parts_max(ws.part, gridDim.x, T_MAX, redu);
    if (threadIdx.x == 0) {
      // Truncated MGS (Algorithm 1, inner loop) from the dots: with
      // v_i = alpha_i v_hat_i and w_true = alpha_j w,
      // H(i,j) = v_i . (w_true - sum_{l<i} H(l,j) v_l).
      const int t = ws.t;
      const double aj = c->alpha[j];
      double h[T_MAX];
      for (int a = 0; a < win.nw; ++a) {
        const int i = win.lo + a;
        const double ai = c->alpha[i];
        double v = ai * aj * p[a];
        for (int b2 = 0; b2 < a; ++b2) {
          const int l = win.lo + b2;
          v -= h[b2] * ai * c->alpha[l] * c->gram[i][i - l - 1];
        }
        h[a] = v;
        c->hband[j][i - j + t - 1] = v;
      }
      double bound = fabs(aj) * __longlong_as_double((long long)wmx);
      c->coef[0] = aj;
      for (int a = 0; a < win.nw; ++a) {
        const int i = win.lo + a;
        c->coef[1 + a] = h[a] * c->alpha[i];
        bound += fabs(c->coef[1 + a]) * __longlong_as_double((long long)c->vmax[i]);
      }
      c->wmax = wmx;
      c->acc_top = window_top(bound * (1.0 + 1e-12), ws.win_bits);
      c->matvecs += 1;
    }
  }
}

cudaError_t launch_spmv_dots(const WS& ws, CsrDev A, const double* const* vcol, int j, cudaStream_t st) {
  Win win;
  win.lo = j - ws.t + 1 > 0 ? j - ws.t + 1 : 0;
  win.nw = j - win.lo + 1;
  for (int a = 0; a < T_MAX; ++a) win.v[a] = a < win.nw ? vcol[win.lo + a] : nullptr;
  k_spmv_dots<<<grid_rows(A.n, 256, ws.grid_max), 256, 0, st>>>(ws, A, win, j);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Arnoldi step j, part 2: v_hat_{j+1}, ||v_hat_{j+1}||^2, window dots for the
// next step, and S v_hat_{j+1} into the 128-bit accumulators ws.acc.
// Partials per CTA: [0] norm^2, [1..t-1] v_hat_{j+1}.v_hat_{j-d}, [T_MAX] max.
// ---------------------------------------------------------------------------
__global__ void k_update_sketch(WS ws, Win win, double* __restrict__ vnext, int j) {
  Ctl* c = ws.ctl;
  if (c->done) return;
  extern __shared__ unsigned char smem[];
  const int tileR = sketch_tile_rows(ws.zeta);
  double* vals = (double*)smem;
  uint16_t* ent_s = (uint16_t*)(vals + tileR);
  uint16_t* ptr_s = ent_s + tileR * ws.zeta;
  __shared__ unsigned long long redu[32];
  __shared__ double red[32];
  const int top = c->acc_top;
  double cf[T_MAX + 1];
#pragma unroll
  for (int a = 0; a <= T_MAX; ++a) cf[a] = a <= win.nw ? c->coef[a] : 0.0;
  const double* __restrict__ w = ws.Wv;
  const int64_t n = ws.n;
  double nrm = 0.0;
  double cr[T_MAX] = {0.0, 0.0, 0.0, 0.0};  // cr[d] = v_hat_{j+1} . v_hat_{j-d}
  unsigned long long vm = 0ull, lo = 0ull, hi = 0ull;
  const int ncross = ws.t - 1;
  const int ntiles = (int)((n + tileR - 1) / tileR);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * tileR;
    const int ncols = (int)(n - r0 < (int64_t)tileR ? n - r0 : (int64_t)tileR);
    for (int i = threadIdx.x; i < tileR; i += blockDim.x) {
      double v = 0.0;
      if (i < ncols) {
        const int64_t r = r0 + i;
        double wv[T_MAX];
#pragma unroll
        for (int a = 0; a < T_MAX; ++a) wv[a] = a < win.nw ? win.v[a][r] : 0.0;
        v = cf[0] * w[r];
#pragma unroll
        for (int a = 0; a < T_MAX; ++a)
          if (a < win.nw) v = fma(-cf[1 + a], wv[a], v);
        vnext[r] = v;
        nrm = fma(v, v, nrm);
#pragma unroll
        for (int d = 0; d < T_MAX; ++d)
          if (d < ncross && d < win.nw) cr[d] = fma(v, wv[win.nw - 1 - d], cr[d]);
        unsigned long long u = abs_bits(v);
        vm = u > vm ? u : vm;
      }
      vals[i] = v;
    }
    __syncthreads();
    tile_sketch_accumulate(ws, tileR, tile, ncols, vals, ent_s, ptr_s, redu, top, lo, hi);
  }
  if (threadIdx.x < ws.s) atomic_add128(ws.acc + 2 * threadIdx.x, lo, hi);
  nrm = block_sum(nrm, red);
#pragma unroll
  for (int d = 0; d < T_MAX; ++d)
    if (d < ncross) cr[d] = block_sum(cr[d], red);
  vm = block_max_u64(vm, redu);
  if (threadIdx.x == 0) {
    double* pp = ws.part + blockIdx.x * NPART;
    pp[0] = nrm;
    for (int d = 0; d < ncross; ++d) pp[1 + d] = cr[d];
    pp[T_MAX] = __longlong_as_double((long long)vm);
  }
}

int update_grid(const WS& ws) { return grid_tiles(ws, ws.n); }

cudaError_t launch_update_sketch(const WS& ws, const double* const* vcol, double* vnext, int j,
                                 cudaStream_t st) {
  Win win;
  win.lo = j - ws.t + 1 > 0 ? j - ws.t + 1 : 0;
  win.nw = j - win.lo + 1;
  for (int a = 0; a < T_MAX; ++a) win.v[a] = a < win.nw ? vcol[win.lo + a] : nullptr;
  size_t sm = sketch_smem_bytes(ws.zeta);
  static bool attr = false;
  cudaError_t e = set_smem((const void*)k_update_sketch, sketch_smem_bytes(ZETA_MAX), attr);
  if (e != cudaSuccess) return e;
  k_update_sketch<<<update_grid(ws), 512, sm, st>>>(ws, win, vnext, j);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x_trial = x + [U, V(:, 0:j+1)] y' with y'_U = y_tilde(0:kh), y'_V,c = y_tilde(kh+c) alpha_c.
// ---------------------------------------------------------------------------
struct Cols {
  const double* v0;  // column 0 of V (the cycle's residual)
  const double* vs;  // columns 1.. (column c at vs + (c-1)*ldv)
};

__global__ void k_check_gemv(WS ws, const double* __restrict__ U, Cols V, const double* __restrict__ xcur,
                             double* __restrict__ xtrial, int kh, int j) {
  Ctl* c = ws.ctl;
  if (!c->check) return;
  __shared__ double cf[D_MAX];
  __shared__ unsigned long long redu[32];
  const int d = kh + j + 1;
  for (int l = threadIdx.x; l < d; l += blockDim.x)
    cf[l] = l < kh ? ws.ytil[l] : ws.ytil[l] * c->alpha[l - kh];
  __syncthreads();
  const int64_t ld = ws.ldv;
  unsigned long long xm = 0ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ws.n; r += (int64_t)gridDim.x * blockDim.x) {
    double acc = xcur[r];
    for (int l = 0; l < kh; ++l) acc = fma(U[r + l * ld], cf[l], acc);
    acc = fma(V.v0[r], cf[kh], acc);
    for (int cc = 1; cc <= j; ++cc) acc = fma(V.vs[r + (int64_t)(cc - 1) * ld], cf[kh + cc], acc);
    xtrial[r] = acc;
    unsigned long long u = abs_bits(acc);
    xm = u > xm ? u : xm;
  }
  xm = block_max_u64(xm, redu);
  if (threadIdx.x == 0) atomicMax(&c->xmax, xm);
}

cudaError_t launch_check_gemv(const WS& ws, const double* U, const double* const* vcol, const double* xcur,
                              double* xtrial, int kh, int j, cudaStream_t st) {
  Cols V{vcol[0], ws.Vs};
  k_check_gemv<<<grid_rows(ws.n, 256, ws.grid_max), 256, 0, st>>>(ws, U, V, xcur, xtrial, kh, j);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// U_new = [U, V(:, 0:jf)] P' (P' rows for V already scaled by alpha).
// ---------------------------------------------------------------------------
__global__ void k_recycle_gemm(WS ws, const double* __restrict__ U, Cols V, double* __restrict__ Unew, int kh) {
  Ctl* c = ws.ctl;
  const int kp = c->kprime;
  const int d = kh + c->jf;
  if (kp <= 0 || c->jf <= 0) return;
  extern __shared__ double Ps[];  // d x kp, row-major (Ps[l*K_MAX + col])
  for (int i = threadIdx.x; i < d * K_MAX; i += blockDim.x) {
    int l = i / K_MAX, cc = i % K_MAX;
    Ps[i] = cc < kp ? ws.P[l + cc * D_MAX] : 0.0;
  }
  __syncthreads();
  const int64_t ld = ws.ldv;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ws.n; r += (int64_t)gridDim.x * blockDim.x) {
    double acc[K_MAX];
#pragma unroll
    for (int cc = 0; cc < K_MAX; ++cc) acc[cc] = 0.0;
    for (int l = 0; l < d; ++l) {
      double wv;
      if (l < kh) wv = U[r + l * ld];
      else if (l == kh) wv = V.v0[r];
      else wv = V.vs[r + (int64_t)(l - kh - 1) * ld];
      const double* pr = Ps + l * K_MAX;
#pragma unroll
      for (int cc = 0; cc < K_MAX; ++cc)
        if (cc < kp) acc[cc] = fma(wv, pr[cc], acc[cc]);
    }
#pragma unroll
    for (int cc = 0; cc < K_MAX; ++cc)
      if (cc < kp) Unew[r + cc * ld] = acc[cc];
  }
}

cudaError_t launch_recycle_gemm(const WS& ws, const double* U, const double* const* vcol, double* Unew, int kh,
                                cudaStream_t st) {
  Cols V{vcol[0], ws.Vs};
  size_t sm = (size_t)D_MAX * K_MAX * sizeof(double);
  static bool attr = false;
  cudaError_t e = set_smem((const void*)k_recycle_gemm, sm, attr);
  if (e != cudaSuccess) return e;
  k_recycle_gemm<<<grid_rows(ws.n, 128, ws.grid_max * 2), 128, sm, st>>>(ws, U, V, Unew, kh);
  return cudaGetLastError();
}

__global__ void k_spmv(CsrDev A, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.n; r += (int64_t)gridDim.x * blockDim.x)
    y[r] = csr_row_dot(A.rowptr, A.col, A.val, x, r);
}

cudaError_t launch_spmv(CsrDev A, const double* x, double* y, cudaStream_t st) {
  int64_t g = (A.n + 255) / 256;
  if (g > 4096) g = 4096;
  k_spmv<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(A, x, y);
  return cudaGetLastError();
}

}  // namespace sdr
