// Small dense part of each GMRES-SDR step (Algorithm 1, sketched least squares
// and residual control), FP64, one CTA.
//
// The economic QR of SAW = [SAU, SAV(:, 1:j)] is updated one column at a time
// with Householder reflectors held in compact WY form Q = I - Y T Y^T
// (Schreiber & Van Loan): the new column c becomes Q^T c = c - Y (T^T (Y^T c))
// through two matrix-vector products, so the work spreads over all threads
// instead of one reflector at a time.  z = Q^T S r0 is kept up to date as
// reflectors are added; the sketched residual ||S r0 - SAW y|| equals the norm
// of z below the current column.
#include "launch.cuh"
#include "eidot.cuh"

namespace sdr {

constexpr int DT = 768;  // threads of the dense-step CTA (512 and 1024 ran slower)

// ---- fixed-point helpers (see eidot.cuh) ----------------------------------
__device__ __forceinline__ Q52 unpack(unsigned long long b) {
  Q52 q;
  q.hi = (int)(b >> 32);
  q.lo = (unsigned)(b & 0xFFFFFFFFull);
  return q;
}
__device__ __forceinline__ unsigned long long pack(Q52 q) {
  return ((unsigned long long)(unsigned)q.hi << 32) | (unsigned long long)q.lo;
}
__device__ __forceinline__ void warp_reduce_acc(Acc3& a) {
  for (int o = 16; o > 0; o >>= 1) {
    a.hh += __shfl_xor_sync(0xffffffffu, a.hh, o);
    a.mx += __shfl_xor_sync(0xffffffffu, a.mx, o);
    a.my += __shfl_xor_sync(0xffffffffu, a.my, o);
    a.ll += __shfl_xor_sync(0xffffffffu, a.ll, o);
  }
}
// Quantise n values of src (shared) into dst with one common exponent; returns
// that exponent e (x ~ X 2^(e-51)).  Block-wide, synchronising.
__device__ int quant_block(const double* src, Q52* dst, int n, unsigned long long* redu) {
  unsigned long long mb = 0ull;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long u = abs_bits(src[i]);
    mb = u > mb ? u : mb;
  }
  mb = block_max_u64(mb, redu);
  const int emax = bexp_of_bits(mb);
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = q52(src[i], emax, 0);
  __syncthreads();
  return emax - 1022;
}

constexpr int YQ_E = 1;  // every Householder vector has max |v_i| = v_p = 1: exponent 1

struct QrSmem {
  double c[S_MAX];
  double z[S_MAX];
  double u[D_MAX];
  double u2[D_MAX];
  Q52 cq[S_MAX];
  Q52 uq[D_MAX];
  double red[DT];
  unsigned long long redu[32];
};

// Add column c (in sm.c, length s) as column p of SAW's QR.  Updates Y, Yq, T,
// Tq, texp, Rf, tau (global) and sm.z.  Returns the sketched residual
// ||z(p+1:s)||.  The products with Y and T run on the integer pipe.
__device__ double qr_add_column(const WS& ws, int p, QrSmem& sm, int* rank_flag) {
  const int s = ws.s, ld = ws.dmax;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* __restrict__ Y = ws.Y;
  double* __restrict__ T = ws.T;
  const unsigned long long* __restrict__ Yq = ws.Yq;
  const unsigned long long* __restrict__ Tq = ws.Tq;
  // u = Y(:, 0:p)^T c
  const int ec = quant_block(sm.c, sm.cq, s, sm.redu);
  for (int l = wid; l < p; l += nw) {
    Acc3 acc;
    acc.zero();
    for (int i = l + lane; i < s; i += 32) acc.mac(unpack(Yq[i + (int64_t)l * s]), sm.cq[i]);
    warp_reduce_acc(acc);
    if (lane == 0) sm.u[l] = acc_to_double(acc, (YQ_E - 51) + (ec - 51));
  }
  __syncthreads();
  // u2 = T(0:p, 0:p)^T u  (column l of T against u)
  const int eu = quant_block(sm.u, sm.uq, p, sm.redu);
  for (int l = wid; l < p; l += nw) {
    Acc3 acc;
    acc.zero();
    for (int m = lane; m <= l; m += 32) acc.mac(unpack(Tq[m + (int64_t)l * ld]), sm.uq[m]);
    warp_reduce_acc(acc);
    if (lane == 0) sm.u2[l] = acc_to_double(acc, (ws.texp[l] - 51) + (eu - 51));
  }
  __syncthreads();
  // c = c - Y u2   (Y(i, l) = 0 for i < l)
  const int eu2 = quant_block(sm.u2, sm.uq, p, sm.redu);
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const int lmax = i < p - 1 ? i : p - 1;
    Acc3 acc;
    acc.zero();
    for (int l = 0; l <= lmax; ++l) acc.mac(unpack(Yq[i + (int64_t)l * s]), sm.uq[l]);
    sm.c[i] -= acc_to_double(acc, (YQ_E - 51) + (eu2 - 51));
  }
  __syncthreads();
  // Householder reflector for c(p:s): H c(p:s) = beta e_1, H = I - tau v v^T, v_0 = 1
  double xs = 0.0;
  for (int i = p + 1 + threadIdx.x; i < s; i += blockDim.x) xs = fma(sm.c[i], sm.c[i], xs);
  xs = block_sum_lean(xs, sm.red);
  const double alpha = sm.c[p];
  double beta, tau, scale;
  if (xs == 0.0) {
    beta = alpha;
    tau = 0.0;
    scale = 0.0;
  } else {
    beta = -copysign(sqrt(alpha * alpha + xs), alpha);
    tau = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
  }
  if (beta == 0.0 && threadIdx.x == 0) *rank_flag = 1;
  // R(0:p, p) = c(0:p), R(p, p) = beta; Y(:, p) = v (|v_i| <= 1, v_p = 1)
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    if (i < p) ws.Rf[i + (int64_t)p * ld] = sm.c[i];
    if (i == p) ws.Rf[i + (int64_t)p * ld] = beta;
    const double v = i < p ? 0.0 : (i == p ? 1.0 : sm.c[i] * scale);
    Y[i + (int64_t)p * s] = v;
    const Q52 q = q52(v, 1022 + YQ_E, 0);
    ws.Yq[i + (int64_t)p * s] = pack(q);
    sm.cq[i] = q;
    sm.c[i] = v;  // c now holds v
  }
  if (threadIdx.x == 0) ws.tau[p] = tau;
  __syncthreads();
  // g = Y(:, 0:p)^T v  (v is zero above p), then T(0:p, p) = -tau T(0:p, 0:p) g
  for (int m = wid; m < p; m += nw) {
    Acc3 acc;
    acc.zero();
    for (int i = p + lane; i < s; i += 32) acc.mac(unpack(Yq[i + (int64_t)m * s]), sm.cq[i]);
    warp_reduce_acc(acc);
    // g_m 2^(texp[m]): column m of T is stored scaled by 2^(-texp[m])
    if (lane == 0) sm.u[m] = acc_to_double(acc, (YQ_E - 51) + (YQ_E - 51) + ws.texp[m]);
  }
  __syncthreads();
  const int eg = quant_block(sm.u, sm.uq, p, sm.redu);
  for (int l = wid; l < p; l += nw) {
    Acc3 acc;
    acc.zero();
    for (int m = l + lane; m < p; m += 32) acc.mac(unpack(Tq[l + (int64_t)m * ld]), sm.uq[m]);
    warp_reduce_acc(acc);
    if (lane == 0) sm.u2[l] = -tau * acc_to_double(acc, -51 + (eg - 51));
  }
  __syncthreads();
  if (threadIdx.x == 0) sm.u2[p] = tau;
  __syncthreads();
  for (int l = threadIdx.x; l <= p; l += blockDim.x) T[l + (int64_t)p * ld] = sm.u2[l];
  const int et = quant_block(sm.u2, sm.uq, p + 1, sm.redu);
  for (int l = threadIdx.x; l <= p; l += blockDim.x) ws.Tq[l + (int64_t)p * ld] = pack(sm.uq[l]);
  if (threadIdx.x == 0) ws.texp[p] = et;
  // z(p:s) -= tau v (v^T z(p:s))
  double dz = 0.0;
  for (int i = p + threadIdx.x; i < s; i += blockDim.x) dz = fma(sm.c[i], sm.z[i], dz);
  dz = block_sum_lean(dz, sm.red);
  for (int i = p + threadIdx.x; i < s; i += blockDim.x) sm.z[i] = fma(-tau * dz, sm.c[i], sm.z[i]);
  __syncthreads();
  double rr = 0.0;
  for (int i = p + 1 + threadIdx.x; i < s; i += blockDim.x) rr = fma(sm.z[i], sm.z[i], rr);
  rr = block_sum_lean(rr, sm.red);
  return sqrt(rr);
}

// ---------------------------------------------------------------------------
// Cycle start (Algorithm 1, before the Arnoldi loop), in two kernels.
// k_cycle_head (Arnoldi stream): S r0 from the residual accumulators,
// beta = ||r0||, the scale of V(:,1), SV(:,1), z = S r0 and the control flags.
// k_cycle_qr (control stream): the QR of the kh recycled columns SAU, which
// only the dense steps need, so the first Arnoldi steps run beside it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DT) k_cycle_head(WS ws, int kh, unsigned long long* accR, int persist_safety) {
  Ctl* c = ws.ctl;
  const int s = ws.s;
  const double beta = c->res;
  const int top = c->accR_top;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double v = int128_to_double(accR[2 * i], accR[2 * i + 1], top - 126) * ws.inv_sqrt_zeta;
    accR[2 * i] = 0ull;
    accR[2 * i + 1] = 0ull;
    ws.Sr0[i] = v;
    ws.z[i] = v;
    ws.SV[i] = beta > 0.0 ? v / beta : 0.0;
  }
  if (threadIdx.x == 0) {
    c->alpha[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    c->vmax[0] = c->rmax;
    c->beta = beta;
    c->kh = kh;
    c->check = 0;
    c->jf = 0;
    c->step = 0;
    c->nchecks = 0;
    c->breakdown = 0;
    c->bd_dense = 0;
    c->rankfail = 0;
    c->tc_error = 0;
    c->kprime = 0;
    c->ell = 0;
    c->svd_path = 0;
    if (!persist_safety) c->safety = c->safety0;
    c->converged = beta < c->tol ? 1 : 0;
    c->done = c->converged;
    c->jstop = c->converged ? -(1 << 20) : (1 << 20);
  }
}

__global__ void __launch_bounds__(DT) k_cycle_qr(WS ws, const double* __restrict__ SAU, int kh) {
  __shared__ QrSmem sm;
  __shared__ int rank_flag;
  Ctl* c = ws.ctl;
  const int s = ws.s;
  if (threadIdx.x == 0) rank_flag = 0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) sm.z[i] = ws.z[i];
  __syncthreads();
  double sres = 0.0;
  {
    double rr = 0.0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) rr = fma(sm.z[i], sm.z[i], rr);
    sres = sqrt(block_sum(rr, sm.red));
  }
  for (int p = 0; p < kh; ++p) {
    for (int i = threadIdx.x; i < s; i += blockDim.x) sm.c[i] = SAU[i + (int64_t)p * s];
    __syncthreads();
    sres = qr_add_column(ws, p, sm, &rank_flag);
  }
  for (int i = threadIdx.x; i < s; i += blockDim.x) ws.z[i] = sm.z[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    c->sres = sres;
    if (rank_flag) c->rankfail = 1;
  }
}

cudaError_t launch_cycle_head(const WS& ws, int kh, unsigned long long* accR, int persist_safety, cudaStream_t st) {
  k_cycle_head<<<1, DT, 0, st>>>(ws, kh, accR, persist_safety);
  return cudaGetLastError();
}

cudaError_t launch_cycle_qr(const WS& ws, const double* SAU, int kh, cudaStream_t st) {
  k_cycle_qr<<<1, DT, 0, st>>>(ws, SAU, kh);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Arnoldi step j, dense part.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(DT) k_step_dense(WS ws, int j, int kh, int ubuf, int grid2, unsigned long long* accR) {
  Ctl* c = ws.ctl;
  if (c->done) return;
  __shared__ QrSmem sm;
  __shared__ double hcol[T_MAX + 1];
  __shared__ double sh_alpha;
  __shared__ int rank_flag;
  __shared__ unsigned long long redu[32];
  const int s = ws.s, t = ws.t;
  const int p = kh + j;
  const int lo = j - t + 1 > 0 ? j - t + 1 : 0;
  // 1. column j+1 was finished (h(j+1, j), alpha_{j+1}) by the kernel that
  //    sketched it
  const bool breakdown = !(c->alpha[j + 1] > 0.0);
  if (threadIdx.x == 0) {
    rank_flag = 0;
    sh_alpha = c->alpha[j + 1];
    for (int o = 0; o <= T_MAX; ++o) hcol[o] = o <= t ? c->hband[j][o] : 0.0;
    c->bd_dense = breakdown ? 1 : 0;
    if (breakdown) {
      hcol[t] = 0.0;
      c->breakdown = 1;
    }
  }
  __syncthreads();
  // 2. S v_hat_{j+1} from the accumulators; SV(:, j+1); 3. SAV(:, j)
  const int top = c->vtop[j + 1];
  const double a1 = sh_alpha;
  unsigned long long* __restrict__ acc = ws.accV + (int64_t)(j + 1) * 2 * S_MAX;  // S v_hat_{j+1}
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double raw = int128_to_double(acc[2 * i], acc[2 * i + 1], top - 126) * ws.inv_sqrt_zeta;
    acc[2 * i] = 0ull;
    acc[2 * i + 1] = 0ull;
    if (breakdown) raw = 0.0;
    ws.SV[i + (int64_t)(j + 1) * s] = raw * a1;
    // SAV(:, j) = SV(:, 1:j+1) H(1:j+1, j) over the band; H(j+1,j) SV(:,j+1) = raw
    double v = raw;
    for (int ii = lo; ii <= j; ++ii) v = fma(hcol[ii - j + t - 1], ws.SV[i + (int64_t)ii * s], v);
    ws.SAV[i + (int64_t)j * s] = v;
    sm.c[i] = v;
    sm.z[i] = ws.z[i];
  }
  __syncthreads();
  // 4. QR update
  const double sres_prev = c->sres;  // ||S r_{j-1}|| = ||z(p:s)||, kept by the previous step
  const double sres = qr_add_column(ws, p, sm, &rank_flag);
  for (int i = threadIdx.x; i < s; i += blockDim.x) ws.z[i] = sm.z[i];
  // 5. residual control (Algorithm 1): check the true residual when
  //    sres < tol / safety, at the last step, or after a breakdown.
  __shared__ int do_check;
  if (threadIdx.x == 0) {
    if (c->hist_n < HIST_MAX) {
      ws.hist[c->hist_n] = sres;
      // Givens sine and cosine of this step (Section 4.5, Theorem on Givens
      // sines; Section 5): the reflector of column p maps z(p:s), of norm
      // ||S r_{j-1}||, to (z_p, z(p+1:s)); a Givens QR of the whitened
      // Hessenberg matrix produces the same pair, |c| = |z_p| / ||S r_{j-1}||
      // and |s| = ||S r_j|| / ||S r_{j-1}||
      const bool ok = sres_prev > 0.0;
      ws.hist_givens[2 * c->hist_n] = ok ? sres / sres_prev : 0.0;
      ws.hist_givens[2 * c->hist_n + 1] = ok ? fabs(sm.z[p]) / sres_prev : 0.0;
    }
    c->hist_n += 1;
    c->sres = sres;
    c->step = j + 1;
    atomicAdd(&c->sketches, 1);
    if (rank_flag) c->rankfail = 1;
    do_check = (sres < c->tol / c->safety) || (j == ws.m - 1) || breakdown;
    c->check = do_check;
    if (do_check) c->xmax = 0ull;
  }
  __syncthreads();
  if (!do_check) return;
  for (int i = threadIdx.x; i < 2 * s; i += blockDim.x) accR[i] = 0ull;
  // y_tilde = R(0:p+1, 0:p+1)^{-1} z(0:p+1) by column-oriented back substitution.
  // The reciprocals of the diagonal are formed in parallel first (an FP64
  // division is a long sequence on this GPU); then one warp runs the
  // substitution, each lane owning rows lane + 32 q and loading the next
  // column of R while the current one is applied.
  double* invd = sm.u2;  // D_MAX doubles, free at this point
  for (int i = threadIdx.x; i <= p; i += blockDim.x) {
    const double rii = ws.Rf[i + (int64_t)i * ws.dmax];
    const bool ok = rii != 0.0 && isfinite(rii);
    invd[i] = ok ? 1.0 / rii : 0.0;
    if (!ok) c->rankfail = 1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    constexpr int NQ = (D_MAX + 31) / 32;
    const double* __restrict__ Rf = ws.Rf;
    const int64_t ldr = ws.dmax;
    double cur[NQ], nxt[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int l = lane + 32 * q;
      cur[q] = l < p ? Rf[l + (int64_t)p * ldr] : 0.0;
    }
    for (int i = p; i >= 0; --i) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int l = lane + 32 * q;
        nxt[q] = (i >= 1 && l < i - 1) ? Rf[l + (int64_t)(i - 1) * ldr] : 0.0;
      }
      __syncwarp();
      const double y = sm.z[i] * invd[i];
      if (lane == 0) ws.ytil[i] = y;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int l = lane + 32 * q;
        if (l < i) sm.z[l] = fma(-cur[q], y, sm.z[l]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) cur[q] = nxt[q];
    }
  }
  __syncthreads();
  // fixed-point coefficients for the check GEMV: y''_l = y'_l 2^(E_l) with
  // y'_l = y_l (U part) or y_l alpha_l (V part) and 2^(-E_l) the column scale
  unsigned long long mb = 0ull;
  for (int l = threadIdx.x; l <= p; l += blockDim.x) {
    const unsigned long long cb = l < kh ? c->umax[ubuf][l] : c->vmax[l - kh];
    const int ce = bexp_of_bits(cb);
    const double yp = l < kh ? ws.ytil[l] : ws.ytil[l] * c->alpha[l - kh];
    const double yy = ce == 0 ? 0.0 : ldexp(yp, ce - 1022);
    sm.c[l] = yy;
    const unsigned long long u = abs_bits(yy);
    mb = u > mb ? u : mb;
  }
  mb = block_max_u64(mb, redu);
  const int emax = bexp_of_bits(mb);
  for (int l = threadIdx.x; l <= p; l += blockDim.x) {
    const Q52 q = q52(sm.c[l], emax, 0);
    ws.ytq[l] = ((unsigned long long)(unsigned)q.hi << 32) | (unsigned long long)q.lo;
  }
  if (threadIdx.x == 0) ws.yexp[0] = emax - 1022;
}

// max |U(:, l)| per column into ctl->umax[ubuf][l].
template <typename T>
__global__ void k_umax(WS ws, const T* __restrict__ U, int kdim, int ubuf) {
  __shared__ unsigned long long redu[32];
  const int l = blockIdx.y;
  unsigned long long m = 0ull;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ws.n; r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long u = abs_bits((double)U[r + (int64_t)l * ws.ldv]);
    m = u > m ? u : m;
  }
  m = block_max_u64(m, redu);
  if (threadIdx.x == 0 && m) atomicMax(&ws.ctl->umax[ubuf][l], m);
}

template <typename T>
cudaError_t launch_umax(const WS& ws, const T* U, int kdim, int ubuf, cudaStream_t st) {
  if (kdim <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(&ws.ctl->umax[ubuf][0], 0, sizeof(unsigned long long) * K_MAX, st);
  if (e != cudaSuccess) return e;
  int gx = (int)((ws.n + 255) / 256);
  if (gx > 64) gx = 64;
  k_umax<T><<<dim3(gx, kdim), 256, 0, st>>>(ws, U, kdim, ubuf);
  return cudaGetLastError();
}

template cudaError_t launch_umax<double>(const WS&, const double*, int, int, cudaStream_t);
template cudaError_t launch_umax<float>(const WS&, const float*, int, int, cudaStream_t);

cudaError_t launch_step_dense(const WS& ws, int j, int kh, int ubuf, unsigned long long* accR, cudaStream_t st) {
  k_step_dense<<<1, DT, 0, st>>>(ws, j, kh, ubuf, update_grid(ws), accR);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Numerical rank of the sketched recycle block SAU (s x kd), for the calls that
// install a recycle space (sdr_recycle, sdr_recycle_import).  Algorithm 1
// solves its least squares problem through R^{-1} of the QR of SAW =
// [SAU, SAV], which needs SAU of full column rank.  Gram-Schmidt with one
// re-orthogonalisation pass gives the diagonal |R_pp| of that QR; the block
// counts as rank-deficient when some |R_pp| <= s * eps * max_q ||SAU(:, q)||
// (or a value is not finite).  One CTA; Q (s x kd) in dynamic shared memory.
// ---------------------------------------------------------------------------
constexpr int RK_T = 512;
__global__ void __launch_bounds__(RK_T) k_sau_rank(const double* __restrict__ SAU, int s, int kd, int* flag) {
  extern __shared__ double rk_dyn[];
  double* Q = rk_dyn;                  // s x kd, column-major
  double* c = Q + (size_t)s * kd;      // the column being reduced
  __shared__ double dots[K_MAX];
  __shared__ double red[RK_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double maxn = 0.0;
  bool bad = false;
  for (int q = 0; q < kd; ++q) {
    double a = 0.0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      const double v = SAU[i + (int64_t)q * s];
      a = fma(v, v, a);
    }
    a = block_sum(a, red);
    if (!isfinite(a)) bad = true;
    maxn = fmax(maxn, sqrt(a));
  }
  const double thresh = (double)s * 2.220446049250313e-16 * maxn;
  for (int p = 0; p < kd && !bad; ++p) {
    for (int i = threadIdx.x; i < s; i += blockDim.x) c[i] = SAU[i + (int64_t)p * s];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = wid; q < p; q += nw) {  // dots[q] = Q(:, q) . c, one warp per column
        double d = 0.0;
        for (int i = lane; i < s; i += 32) d = fma(Q[i + (size_t)q * s], c[i], d);
        d = warp_sum(d);
        if (lane == 0) dots[q] = d;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < s; i += blockDim.x) {
        double v = c[i];
        for (int q = 0; q < p; ++q) v = fma(-dots[q], Q[i + (size_t)q * s], v);
        c[i] = v;
      }
      __syncthreads();
    }
    double rr = 0.0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) rr = fma(c[i], c[i], rr);
    const double rpp = sqrt(block_sum(rr, red));
    if (!(rpp > thresh)) bad = true;  // uniform: every thread holds the same rpp
    const double inv = rpp > 0.0 ? 1.0 / rpp : 0.0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) Q[i + (size_t)p * s] = c[i] * inv;
    __syncthreads();
  }
  if (threadIdx.x == 0) *flag = (bad || !(maxn > 0.0)) ? 1 : 0;
}

cudaError_t launch_sau_rank(const double* SAU, int s, int kd, int* flag, cudaStream_t st) {
  const size_t smem = ((size_t)s * kd + s) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_sau_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_sau_rank<<<1, RK_T, smem, st>>>(SAU, s, kd, flag);
  return cudaGetLastError();
}

}  // namespace sdr
