// Cycle end of GMRES-SDR: sketched harmonic-Ritz update of the recycle space
// (Section 3.5 and the last block of Algorithm 1), FP64.
//
// With SAW = Q R (the QR kept by the step kernels) and S[U V] the sketched
// basis, the sketched harmonic Ritz problem is M y = mu y with
// M = (SAW)^+ S[U V] = R^{-1} (Q^T S[U V]) when SAW has full numerical rank;
// mu = 1/theta and the k largest |mu| are kept.  The paper regularises with a
// truncated SVD SAW ~ U_l S_l V_l^* and takes QZ of (M_l, S_l) with
// M_l = U_l^* S[U V] V_l.  When ell = d the two give the same eigenpairs (they
// are similar through V_l), so the kernels first certify ell = d cheaply:
//   sigma_min(R) >= 1/||R^{-1}||_F and sigma_max(R) <= ||R||_F, hence
//   ||R||_F ||R^{-1}||_F < 1/(d eps) implies sigma_i > sigma_1 d eps for all i.
// Otherwise a one-sided Jacobi SVD of R gives the truncated problem.
//
// Eigenpairs: FP32 Householder reduction to Hessenberg form and Francis
// double-shift QR for candidate eigenvalues; for each candidate an FP64
// eigenpair of M from FP32 factorisations with FP64 residuals (inverse
// iteration, then the refinement of Dongarra, Moler and Wilkinson); the
// selection of the k largest |mu|, and an orthonormal real basis of the span
// of their eigenvectors (real and imaginary parts of complex pairs).
#include <cooperative_groups.h>

#include "launch.cuh"
#include "eidot.cuh"

namespace sdr {

constexpr int LDD = D_MAX;  // leading dimension of the d x d scratch matrices
constexpr int KC_MARGIN = 8;      // extra eigenvalue candidates beyond k
constexpr int KC = K_MAX + KC_MARGIN + 1;  // candidates refined in FP64

struct CeLayout {
  double *C, *Rinv, *M, *Hc, *Vh, *As, *tauH, *wr, *wi, *Zr, *Pu, *colsq, *misc;
  double *cmu, *cref, *cvec;  // candidate estimates, FP64 eigenvalues, FP64 vectors (re, im)
  int* sel;   // [K_MAX] eigenvalue index per inverse iteration
  int* zcol;  // [K_MAX] first Z column of that eigenvalue
  int* cnt;   // [0] number of inverse iterations
  int* ivfail;  // [KC] candidate left to the FP64 fallback
  double* lu;   // KC blocks of 2*LDD*LDD (the fallback's complex LU)
  float* H32;   // LDD x LDD: k_ce_eig's FP32 Hessenberg form of M with its reflectors below the subdiagonal
};

__host__ __device__ inline CeLayout ce_layout(double* base) {
  CeLayout L;
  const int64_t dd = (int64_t)LDD * LDD;
  L.C = base;
  L.Rinv = L.C + dd;
  L.M = L.Rinv + dd;
  L.Hc = L.M + dd;
  L.Vh = L.Hc + dd;
  L.As = L.Vh + dd;
  L.tauH = L.As + dd;
  L.wr = L.tauH + LDD;
  L.wi = L.wr + LDD;
  L.Zr = L.wi + LDD;
  L.Pu = L.Zr + (int64_t)LDD * K_MAX;
  L.colsq = L.Pu + (int64_t)LDD * K_MAX;
  L.misc = L.colsq + 2 * LDD;
  L.sel = (int*)(L.misc + 64);
  L.zcol = L.sel + K_MAX;
  L.cnt = L.zcol + K_MAX;
  L.cmu = L.misc + 64 + 3 * K_MAX;
  L.cref = L.cmu + 2 * KC;
  L.cvec = L.cref + 2 * KC;
  L.ivfail = L.cnt + K_MAX;  // inside the 3 K_MAX doubles reserved after misc (6 K_MAX ints, KC <= 3 K_MAX)
  L.lu = L.cvec + (int64_t)2 * KC * LDD;
  L.H32 = (float*)(L.lu + (int64_t)KC * 2 * LDD * LDD);
  return L;
}

size_t ce_scratch_doubles() {
  return (size_t)6 * LDD * LDD + 3 * LDD + 2 * (size_t)LDD * K_MAX + 2 * LDD + 64 + 3 * K_MAX + 4 * KC +
         (size_t)2 * KC * LDD + (size_t)KC * 2 * LDD * LDD + (size_t)LDD * LDD / 2 + 64;
}

// Column l of S[U V] / SAW (sketched basis / sketched image).
__device__ inline const double* sv_col(const WS& ws, const double* SU, int kh, int l) {
  return l < kh ? SU + (int64_t)l * ws.s : ws.SV + (int64_t)(l - kh) * ws.s;
}
__device__ inline const double* saw_col(const WS& ws, const double* SAU, int kh, int l) {
  return l < kh ? SAU + (int64_t)l * ws.s : ws.SAV + (int64_t)(l - kh) * ws.s;
}

// ---------------------------------------------------------------------------
// C(:, col) = (Q^T S[U V](:, col))(0:d);  colsq[col] = ||R(:, col)||^2.
// ---------------------------------------------------------------------------
__global__ void k_ce_formC(WS ws, const double* __restrict__ SU, int kh) {
  Ctl* c = ws.ctl;
  const int d = kh + c->jf;
  const int col = blockIdx.x;
  if (c->jf <= 0 || col >= d) return;
  CeLayout L = ce_layout(ws.dscr);
  __shared__ double x[S_MAX], u[D_MAX], u2[D_MAX], red[32];
  const int s = ws.s, ld = ws.dmax;
  const double* src = sv_col(ws, SU, kh, col);
  for (int i = threadIdx.x; i < s; i += blockDim.x) x[i] = src[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = wid; l < d; l += nw) {
    const double* yc = ws.Y + (int64_t)l * s;
    double a = 0.0;
    for (int i = l + lane; i < s; i += 32) a = fma(yc[i], x[i], a);
    a = warp_sum(a);
    if (lane == 0) u[l] = a;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < d; l += blockDim.x) {
    const double* tc = ws.T + (int64_t)l * ld;
    double a = 0.0;
    for (int m = 0; m <= l; ++m) a = fma(tc[m], u[m], a);
    u2[l] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    double a = x[i];
    for (int l = 0; l <= i; ++l) a = fma(-ws.Y[i + (int64_t)l * s], u2[l], a);
    L.C[i + (int64_t)col * LDD] = a;
  }
  double rs = 0.0;
  for (int i = threadIdx.x; i <= col; i += blockDim.x) {
    const double v = ws.Rf[i + (int64_t)col * ld];
    rs = fma(v, v, rs);
  }
  rs = block_sum(rs, red);
  if (threadIdx.x == 0) L.colsq[col] = rs;
}

// R^{-1}(:, col) by column-oriented back substitution (one warp per column).
__global__ void k_ce_rinv(WS ws, int kh) {
  Ctl* c = ws.ctl;
  const int d = kh + c->jf;
  const int col = blockIdx.x;
  if (c->jf <= 0 || col >= d) return;
  CeLayout L = ce_layout(ws.dscr);
  __shared__ double y[D_MAX];
  const int ld = ws.dmax;
  for (int i = threadIdx.x; i < d; i += blockDim.x) y[i] = (i == col) ? 1.0 : 0.0;
  __syncwarp();
  bool bad = false;
  for (int i = col; i >= 0; --i) {
    const double rii = ws.Rf[i + (int64_t)i * ld];
    const double yi = (rii != 0.0) ? y[i] / rii : 0.0;
    bad |= !(rii != 0.0);
    __syncwarp();
    if (threadIdx.x == 0) y[i] = yi;
    for (int l = threadIdx.x; l < i; l += 32) y[l] = fma(-ws.Rf[l + (int64_t)i * ld], yi, y[l]);
    __syncwarp();
  }
  double ss = 0.0;
  for (int i = threadIdx.x; i < d; i += 32) {
    L.Rinv[i + (int64_t)col * LDD] = y[i];
    ss = fma(y[i], y[i], ss);
  }
  ss = warp_sum(ss);
  if (threadIdx.x == 0) L.colsq[LDD + col] = bad ? INFINITY : ss;
}

// Certificate of full numerical rank and M = R^{-1} C (columns in parallel).
__global__ void k_ce_M(WS ws, int kh) {
  Ctl* c = ws.ctl;
  const int d = kh + c->jf;
  const int col = blockIdx.x;
  if (c->jf <= 0 || col >= d) return;
  CeLayout L = ce_layout(ws.dscr);
  __shared__ int certified;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < d; ++i) {
      a += L.colsq[i];
      b += L.colsq[LDD + i];
    }
    const double prod = sqrt(a) * sqrt(b);
    const double eps = 2.220446049250313e-16;
    certified = (isfinite(prod) && prod * (double)d * eps * 1.001 < 1.0 && !c->force_svd) ? 1 : 0;
    if (col == 0) {
      c->svd_path = certified ? 0 : 1;
      c->ell = certified ? d : 0;
    }
  }
  __syncthreads();
  if (!certified) return;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    double a = 0.0;
    for (int l = i; l < d; ++l) a = fma(L.Rinv[i + (int64_t)l * LDD], L.C[l + (int64_t)col * LDD], a);
    L.M[i + (int64_t)col * LDD] = a;
  }
}

// ---------------------------------------------------------------------------
// Truncated-SVD path: one-sided Jacobi (Hestenes) on R, then
// M_l = S_l^{-1} U_l^T C V_l and V_l kept for P = V_l Z.
//
// The rotations run on a cluster of SVD_CTAS CTAs (one per SM, so the FP64
// pipes of all of them work).  The pairs of a round are dealt out to the
// CTAs, and each pair gets all the warps of its CTA that the round leaves
// free: each warp handles a slice of the two columns, the warps' partial dot
// products are combined in shared memory, one thread forms the rotation, and
// the slices are rotated in parallel.  Column c of the working matrix and of V lives
// in the shared memory of CTA c mod SVD_CTAS and is reached by every CTA of
// the cluster through distributed shared memory.  In each round of the
// round-robin ordering the d/2 disjoint column pairs are spread over all
// warps of the cluster, and a cluster barrier separates the rounds.  A pair
// is rotated when |a_p . a_q| > d eps ||a_p|| ||a_q|| (the one-sided Jacobi
// threshold) and neither column has fallen below the truncation level; the
// sweeps stop when a sweep rotates nothing.  Each sweep visits the columns in
// order of decreasing norm (de Rijk's ordering), which cuts the number of
// sweeps.
// ---------------------------------------------------------------------------
constexpr int SVD_CTAS = 8;
constexpr int SVD_COLS = (D_MAX + SVD_CTAS - 1) / SVD_CTAS;  // columns per CTA

size_t ce_svd_smem() { return (size_t)2 * SVD_COLS * LDD * sizeof(double); }

__global__ void __launch_bounds__(512) k_ce_svd(WS ws, int kh) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0 || !c->svd_path) return;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int d = kh + c->jf;
  CeLayout L = ce_layout(ws.dscr);
  extern __shared__ __align__(16) double svd_sm[];
  double* Aloc = svd_sm;                       // [SVD_COLS][LDD]: columns rank, rank + SVD_CTAS, ...
  double* Vloc = svd_sm + SVD_COLS * LDD;
  __shared__ double sig[D_MAX];
  __shared__ int order[D_MAX];
  __shared__ unsigned long long redu[32];
  __shared__ int sweep_flag[2];                // rank 0's copy: a rotation happened in that sweep
  __shared__ double cnorm[D_MAX];              // rank 0's copy: squared column norms at a sweep's start
  __shared__ int perm[D_MAX];                  // visiting order of the sweep (rank 0's copy, then local)
  __shared__ double wpart[16 * 3];             // per-warp partial dots of a round
  __shared__ double rotp[16 * 2];              // per-pair rotation (cs, sn) of a round
  __shared__ int rotf[16];                     // per-pair: rotate in this round
  const int ld = ws.dmax;
  for (int idx = threadIdx.x; idx < SVD_COLS * d; idx += blockDim.x) {
    const int q = idx / d, i = idx % d;
    const int col = rank + q * SVD_CTAS;
    if (col < d) {
      Aloc[q * LDD + i] = i <= col ? ws.Rf[i + (int64_t)col * ld] : 0.0;
      Vloc[q * LDD + i] = i == col ? 1.0 : 0.0;
    }
  }
  // largest column norm of R: sigma_1 lies within a factor sqrt(d) of it
  double cm = 0.0;
  for (int jj = threadIdx.x; jj < d; jj += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i <= jj; ++i) a = fma(ws.Rf[i + (int64_t)jj * ld], ws.Rf[i + (int64_t)jj * ld], a);
    cm = a > cm ? a : cm;
  }
  cm = __longlong_as_double((long long)block_max_u64((unsigned long long)__double_as_longlong(cm), redu));
  const double eps = 2.220446049250313e-16;
  const double tol = (double)d * eps;
  const double negl = cm * tol * tol;  // squared norm below which a column is treated as zero (truncation level)
  if (threadIdx.x < 2) sweep_flag[threadIdx.x] = 0;
  cluster.sync();
  int* flag0 = cluster.map_shared_rank(&sweep_flag[0], 0);
  auto colA = [&](int col) { return cluster.map_shared_rank(Aloc, col % SVD_CTAS) + (col / SVD_CTAS) * LDD; };
  auto colV = [&](int col) { return cluster.map_shared_rank(Vloc, col % SVD_CTAS) + (col / SVD_CTAS) * LDD; };
  const int dd = d + (d & 1);  // even number of players; index d (if odd) is a dummy
  const int lane = threadIdx.x & 31;
  int sweeps = 0;
  double* cnorm0 = cluster.map_shared_rank(cnorm, 0);
  int* perm0 = cluster.map_shared_rank(perm, 0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    const int par = sweep & 1;
    int rotated = 0;
    // de Rijk: order the columns by decreasing norm (ties by index)
    for (int q = threadIdx.x >> 5; q < SVD_COLS; q += blockDim.x >> 5) {
      const int col = rank + q * SVD_CTAS;
      if (col < d) {
        double a = 0.0;
        for (int i = lane; i < d; i += 32) a = fma(Aloc[q * LDD + i], Aloc[q * LDD + i], a);
        a = warp_sum(a);
        if (lane == 0) cnorm0[col] = a;
      }
    }
    cluster.sync();
    if (rank == 0) {
      // squared norms are >= 0, whose bit patterns order like the values (an
      // integer compare keeps the FP64 pipe free)
      const long long* cb = (const long long*)cnorm;
      for (int i = threadIdx.x; i < d; i += blockDim.x) {
        const long long ni = cb[i];
        int r = 0;
        for (int j2 = 0; j2 < d; ++j2) {
          const long long nj = cb[j2];
          r += (nj > ni || (nj == ni && j2 < i)) ? 1 : 0;
        }
        perm[r] = i;
      }
    }
    cluster.sync();
    if (rank != 0)
      for (int i = threadIdx.x; i < d; i += blockDim.x) perm[i] = perm0[i];
    __syncthreads();
    for (int round = 0; round < dd - 1; ++round) {
      // pairs k = rank, rank + SVD_CTAS, ... of this round belong to this CTA;
      // each gets wpp warps, warp `part` of a pair takes elements
      // part*32 + lane + 32*wpp*it
      const int npc = (dd / 2 - rank + SVD_CTAS - 1) / SVD_CTAS;  // pairs of this CTA (>= 0)
      const int nwarp = blockDim.x >> 5;
      const int wpp = npc > 0 ? (nwarp / npc > 0 ? nwarp / npc : 1) : 1;
      const int w = threadIdx.x >> 5;
      const int q = w / wpp, part = w % wpp;
      int a = 0, b = d;
      const int k = rank + q * SVD_CTAS;
      if (q < npc && k < dd / 2) {
        if (k == 0) {
          a = 0;
          b = 1 + (round % (dd - 1));
        } else {
          a = 1 + ((k + round) % (dd - 1));
          b = 1 + ((dd - 1 - k + round) % (dd - 1));
        }
        if (a > b) { int tmp = a; a = b; b = tmp; }
      }
      const bool live = b < d && q < npc;
      if (live) {
        a = perm[a];
        b = perm[b];
      } else {
        a = 0;
        b = 0;
      }
      double* ap = colA(a);
      double* aq = colA(b);
      double* vp = colV(a);
      double* vq = colV(b);
      constexpr int NE = (D_MAX + 31) / 32;  // elements per lane when one warp holds a pair
      double xa[NE], xb[NE], ya[NE], yb[NE];
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int i = part * 32 + lane + 32 * wpp * u;
        const bool in = live && i < d;
        xa[u] = in ? ap[i] : 0.0;
        xb[u] = in ? aq[i] : 0.0;
        ya[u] = in ? vp[i] : 0.0;
        yb[u] = in ? vq[i] : 0.0;
      }
      double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        if (part * 32 + 32 * wpp * u < d) {  // warp-uniform
          al = fma(xa[u], xa[u], al);
          be = fma(xb[u], xb[u], be);
          ga = fma(xa[u], xb[u], ga);
        }
      }
      // The three butterfly sums (x + partner at distances 16, 8, 4, 2, 1), packed
      // so that lanes which would only repeat a sum work on another of the three:
      // six FP64 adds per warp instead of fifteen (each one holds this warp's
      // FP64 pipe for a full warp's time), with the same additions as three
      // separate butterflies.  al ends in lane 0, ga in lane 8, be in lane 16.
      double s16a, s16b;
      {
        const double own = lane < 16 ? al : be;
        const double snd = lane < 16 ? be : al;
        s16a = own + __shfl_xor_sync(0xffffffffu, snd, 16);  // lanes 0-15: al, 16-31: be
        s16b = ga + __shfl_xor_sync(0xffffffffu, ga, 16);    // lanes 0-15: ga
      }
      double s8;
      {
        const double own = (lane >= 8 && lane < 16) ? s16b : s16a;
        const double snd = lane < 8 ? s16b : s16a;
        s8 = own + __shfl_xor_sync(0xffffffffu, snd, 8);  // lanes 0-7: al, 8-15: ga, 16-23: be
      }
      s8 += __shfl_xor_sync(0xffffffffu, s8, 4);
      s8 += __shfl_xor_sync(0xffffffffu, s8, 2);
      s8 += __shfl_xor_sync(0xffffffffu, s8, 1);
      if (lane == 0) wpart[w * 3 + 0] = s8;
      if (lane == 16) wpart[w * 3 + 1] = s8;
      if (lane == 8) wpart[w * 3 + 2] = s8;
      __syncthreads();
      // the pair's first warp combines the parts and forms the rotation
      if (live && part == 0 && lane == 0) {
        double sa = wpart[w * 3 + 0], sb = wpart[w * 3 + 1], sg = wpart[w * 3 + 2];
        for (int t2 = 1; t2 < wpp; ++t2) {
          sa += wpart[(w + t2) * 3 + 0];
          sb += wpart[(w + t2) * 3 + 1];
          sg += wpart[(w + t2) * 3 + 2];
        }
        // sa, sb, negl >= 0: integer compares of their bit patterns
        const bool big = __double_as_longlong(sa) > __double_as_longlong(negl) &&
                         __double_as_longlong(sb) > __double_as_longlong(negl);
        const bool rot = big && (sg * sg > tol * tol * sa * sb);
        double cs = 1.0, sn = 0.0;
        if (rot) {
          // The rotation angle needs only single precision (an inexact angle
          // still gives an exactly orthogonal rotation, and the next sweep
          // removes what it leaves); the cosine is refined to double
          // precision so that cs^2 + sn^2 = 1 to rounding.  FP64 division and
          // square root are long instruction sequences on this GPU.
          const double num = sb - sa, den = 2.0 * sg;
          const int en = (int)(((unsigned long long)__double_as_longlong(num) >> 52) & 0x7FF);
          const int ed = (int)(((unsigned long long)__double_as_longlong(den) >> 52) & 0x7FF);
          int e = (en > ed ? en : ed) - 1023;
          e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
          const double sc = __longlong_as_double((long long)((unsigned long long)(1023 - e) << 52));
          const float zf = __fdividef((float)(num * sc), (float)(den * sc));
          const float az = fabsf(zf);
          const float tf = az > 1e18f ? copysignf(0.5f / az, zf)
                                      : copysignf(1.0f, zf) / (az + sqrtf(fmaf(zf, zf, 1.0f)));
          const double t = (double)tf;
          // cs = 1 / sqrt(1 + t^2): FP32 estimate, three Newton steps y <- y (3 - x y^2) / 2
          const double xq = fma(t, t, 1.0);
          cs = (double)rsqrtf((float)xq);
#pragma unroll
          for (int it = 0; it < 3; ++it) cs = cs * fma(-0.5 * xq, cs * cs, 1.5);
          sn = cs * t;
        }
        rotp[q * 2 + 0] = cs;
        rotp[q * 2 + 1] = sn;
        rotf[q] = rot ? 1 : 0;
      }
      __syncthreads();
      if (live && rotf[q]) {
        const double cs = rotp[q * 2 + 0], sn = rotp[q * 2 + 1];
#pragma unroll
        for (int u = 0; u < NE; ++u) {
          const int i = part * 32 + lane + 32 * wpp * u;
          if (i < d) {
            ap[i] = cs * xa[u] - sn * xb[u];
            aq[i] = sn * xa[u] + cs * xb[u];
            vp[i] = cs * ya[u] - sn * yb[u];
            vq[i] = sn * ya[u] + cs * yb[u];
          }
        }
        rotated = 1;
      }
      cluster.sync();
    }
    if (rotated && lane == 0) atomicOr(flag0 + par, 1);
    if (rank == 0 && threadIdx.x == 0) sweep_flag[1 - par] = 0;  // the next sweep's flag (nobody reads it yet)
    cluster.sync();
    const int any = *(volatile int*)(flag0 + par);
    cluster.sync();  // every CTA has read the flag before rank 0 clears it in the sweep after next
    sweeps = sweep + 1;
    if (!any) break;
  }
  // every CTA writes its columns back for the rest of the step, run by rank 0
  double* A = L.As;   // working matrix (d x d)
  double* V = L.Vh;   // right singular vectors
  for (int idx = threadIdx.x; idx < SVD_COLS * d; idx += blockDim.x) {
    const int q = idx / d, i = idx % d;
    const int col = rank + q * SVD_CTAS;
    if (col < d) {
      A[i + (int64_t)col * LDD] = Aloc[q * LDD + i];
      V[i + (int64_t)col * LDD] = Vloc[q * LDD + i];
    }
  }
  __threadfence();
  cluster.sync();
  if (rank == 0 && threadIdx.x == 0) c->svd_sweeps = sweeps;
  if (rank != 0) return;
  // singular values and ordering (descending)
  for (int i = threadIdx.x >> 5; i < d; i += blockDim.x >> 5) {
    double a = 0.0;
    for (int r = lane; r < d; r += 32) {
      const double ar = __ldcg(A + r + (int64_t)i * LDD);
      a = fma(ar, ar, a);
    }
    a = warp_sum(a);
    if (lane == 0) sig[i] = sqrt(a);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // singular values are >= 0: integer compares of their bit patterns
    const long long* sgb = (const long long*)sig;
    for (int i = 0; i < d; ++i) order[i] = i;
    for (int i = 1; i < d; ++i) {  // insertion sort, stable
      int v = order[i], y = i - 1;
      while (y >= 0 && sgb[order[y]] < sgb[v]) { order[y + 1] = order[y]; --y; }
      order[y + 1] = v;
    }
    const double s1 = sig[order[0]];
    const long long thr = __double_as_longlong(s1 * (double)d * eps);
    int ell = 0;
    for (int i = 0; i < d; ++i) ell += sgb[order[i]] > thr ? 1 : 0;
    c->ell = ell;
    if (ell == 0) c->rankfail = 1;
  }
  __syncthreads();
  const int ell = c->ell;
  // T1 = C V_l (d x ell) into Hc temporarily; then M = S^{-1} U_l^T T1, U_l = A_l / sigma
  double* T1 = L.Hc;
  for (int idx = threadIdx.x; idx < d * ell; idx += blockDim.x) {
    const int i = idx % d, q = idx / d;
    const double* vc = V + (int64_t)order[q] * LDD;
    double a = 0.0;
    for (int l = 0; l < d; ++l) a = fma(L.C[i + (int64_t)l * LDD], __ldcg(vc + l), a);
    T1[i + (int64_t)q * LDD] = a;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ell * ell; idx += blockDim.x) {
    const int i = idx % ell, q = idx / ell;
    const double si = sig[order[i]];
    const double* uc = A + (int64_t)order[i] * LDD;
    double a = 0.0;
    for (int l = 0; l < d; ++l) a = fma(__ldcg(uc + l), T1[l + (int64_t)q * LDD], a);
    L.M[i + (int64_t)q * LDD] = a / (si * si);  // U_l = A_l / sigma, then S^{-1}
  }
  __syncthreads();
  // keep V_l (ordered) in the columns of As for P = V_l Z
  for (int idx = threadIdx.x; idx < d * ell; idx += blockDim.x) {
    const int i = idx % d, q = idx / d;
    T1[i + (int64_t)q * LDD] = __ldcg(V + i + (int64_t)order[q] * LDD);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < d * ell; idx += blockDim.x) {
    const int i = idx % d, q = idx / d;
    V[i + (int64_t)q * LDD] = T1[i + (int64_t)q * LDD];
  }
}

// ---------------------------------------------------------------------------
// Eigenvalue estimates in FP32: Householder reduction to Hessenberg form and
// Francis double-shift QR, then the candidate list (k + KC_MARGIN largest
// |mu|, conjugate pairs kept whole).  FP32 only locates the eigenvalues; every
// selected eigenpair is recomputed in FP64 by inverse iteration with M itself.
// (On this GPU a full-warp FP64 instruction and a one-lane FP64 instruction
// occupy the FP64 pipe equally, so a sequential FP64 QR sweep on one SM costs
// milliseconds; the FP32 sweep does not.)
// ---------------------------------------------------------------------------
__device__ inline float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float block_sum_f(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_f(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    float r = lane < nw ? red[lane] : 0.f;
    r = warp_sum_f(r);
    if (lane == 0) red[0] = r;
  }
  __syncthreads();
  const float r = red[0];
  __syncthreads();
  return r;
}


// ---------------------------------------------------------------------------
// FP32 eigenvalues of the upper-Hessenberg H by the implicitly double-shifted
// (Francis) QR iteration, as set out in Golub and Van Loan, Matrix
// Computations (4th ed.), Section 7.5: Algorithm 7.5.1 (one Francis step on an
// unreduced Hessenberg block) inside the deflation loop of Algorithm 7.5.2.
// Only the eigenvalues are wanted, so each step transforms the active block
// H(lo:hi, lo:hi) alone.  Reflectors are the Householder vectors of
// Algorithm 5.1.1, v = (1, v1, v2) with P = I - beta v v^T.  Each double-shift
// step starts its bulge at the largest m in [lo, hi-2] where the subdiagonal
// entry H(m, m-1) is small enough that the first reflector's effect on it is
// negligible (Wilkinson, The Algebraic Eigenvalue Problem, on two consecutive
// small subdiagonal elements): starting at lo instead destroys, in FP32, the
// accuracy of eigenvalues of a nearly decoupled leading part.  H is scaled by
// a power of two to a norm of order one first, so that the products in the
// first column of (H - s1 I)(H - s2 I) neither underflow nor overflow.
//
// GPU arrangement (QR_WARPS warps, one named barrier per bulge position):
// at the step whose reflector acts on indices a, a+1, a+2, warp 0 updates the
// neighbourhood of the bulge (rows a..a+2 on columns up to a+3, then columns
// a..a+2 on rows a..a+3) and forms the next reflector, QR_RW warps apply the
// row transformation to columns a+4..hi and QR_CW warps the column
// transformation to rows lo..a-1.  The three parts touch disjoint entries.
// ---------------------------------------------------------------------------
__device__ inline float& HF(float* H, int ldh, int i, int j) { return H[i + j * ldh]; }

constexpr int QR_RW = 2, QR_CW = 2, QR_WARPS = 1 + QR_RW + QR_CW;
__device__ __forceinline__ void qr_bar() { asm volatile("bar.sync 1, %0;" ::"n"(32 * QR_WARPS) : "memory"); }

// Householder vector of (x, y, z) (z = 0 and three = false for a 2-vector):
// P (x, y, z)^T = (mu, 0, 0)^T with P = I - beta v v^T, v = (1, v1, v2).
struct Refl {
  float beta, v1, v2;
};
__device__ __forceinline__ Refl house3(float x, float y, float z) {
  Refl h{0.f, 0.f, 0.f};
  // P depends only on the direction of (x, y, z): scale it to a maximum
  // magnitude of one so that the squares below neither underflow nor overflow
  const float mx = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
  if (!(mx > 0.f) || !isfinite(mx)) return h;
  const float is = 1.f / mx;
  x *= is;
  y *= is;
  z *= is;
  const float sig = y * y + z * z;
  if (sig == 0.f) return h;  // already of the form (x, 0, 0): P = I
  const float mu = sqrtf(x * x + sig);
  const float w = x <= 0.f ? x - mu : -sig / (x + mu);  // the first entry of x - mu e1, without cancellation
  h.v1 = y / w;
  h.v2 = z / w;
  h.beta = 2.f * w * w / (sig + w * w);
  return h;
}

// Left transformation of rows a, a+1 (, a+2) on columns j0 + off + stride t
// <= j1: every load (at most NS columns per thread) is issued before any store.
template <int NS>
__device__ __forceinline__ void refl_rows(float* H, int ldh, int a, bool three, Refl P, int j0, int j1, int off,
                                          int stride) {
  float r0[NS], r1[NS], r2[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int j = j0 + off + stride * t;
    const bool in = j <= j1;
    r0[t] = in ? HF(H, ldh, a, j) : 0.f;
    r1[t] = in ? HF(H, ldh, a + 1, j) : 0.f;
    r2[t] = (in && three) ? HF(H, ldh, a + 2, j) : 0.f;
  }
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int j = j0 + off + stride * t;
    if (j <= j1) {
      const float w = P.beta * (r0[t] + P.v1 * r1[t] + P.v2 * r2[t]);
      HF(H, ldh, a, j) = r0[t] - w;
      HF(H, ldh, a + 1, j) = r1[t] - w * P.v1;
      if (three) HF(H, ldh, a + 2, j) = r2[t] - w * P.v2;
    }
  }
}

// Right transformation of columns a, a+1 (, a+2) on rows i0 + off + stride t <= i1.
template <int NS>
__device__ __forceinline__ void refl_cols(float* H, int ldh, int a, bool three, Refl P, int i0, int i1, int off,
                                          int stride) {
  float c0[NS], c1[NS], c2[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int i = i0 + off + stride * t;
    const bool in = i <= i1;
    c0[t] = in ? HF(H, ldh, i, a) : 0.f;
    c1[t] = in ? HF(H, ldh, i, a + 1) : 0.f;
    c2[t] = (in && three) ? HF(H, ldh, i, a + 2) : 0.f;
  }
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    const int i = i0 + off + stride * t;
    if (i <= i1) {
      const float w = P.beta * (c0[t] + P.v1 * c1[t] + P.v2 * c2[t]);
      HF(H, ldh, i, a) = c0[t] - w;
      HF(H, ldh, i, a + 1) = c1[t] - w * P.v1;
      if (three) HF(H, ldh, i, a + 2) = c2[t] - w * P.v2;
    }
  }
}

// Eigenvalues of the 2 x 2 block [[p, q], [r, s]] from its trace and
// determinant: two real values (the larger-magnitude root first, the other
// from the product) or a conjugate pair.
__device__ __forceinline__ void eig2x2(float p, float q, float r, float s, float& re1, float& im1, float& re2,
                                       float& im2) {
  const float half = 0.5f * (p - s);
  const float disc = half * half + q * r;
  const float mid = 0.5f * (p + s);
  if (disc >= 0.f) {
    const float root = sqrtf(disc);
    const float big = mid + copysignf(root, mid);
    const float det = p * s - q * r;
    re1 = big;
    re2 = big != 0.f ? det / big : mid - root;
    im1 = im2 = 0.f;
  } else {
    const float root = sqrtf(-disc);
    re1 = re2 = mid;
    im1 = root;
    im2 = -root;
  }
}

// Runs on the first QR_WARPS warps of the block; returns false when the
// iteration limit is reached (the eigenvalues not yet found are set to NaN).
// sh: 8 floats of shared memory for passing the next reflector's input.
__device__ bool francis_eigenvalues(float* H, int ldh, int n, float* wr, float* wi, float* sh) {
  const int tid = threadIdx.x, lane = tid & 31, wrp = tid >> 5;
  const float ulp = 1.1920929e-7f;
  float hnorm = 0.f;  // a scale for the deflation test where both diagonal entries vanish
  for (int idx = lane; idx < n * n; idx += 32) {
    const int i = idx % n, j = idx / n;
    if (i <= j + 1) hnorm += fabsf(HF(H, ldh, i, j));
  }
  for (int o = 16; o > 0; o >>= 1) hnorm += __shfl_xor_sync(0xffffffffu, hnorm, o);
  int hexp = 0;
  frexpf(hnorm > 0.f ? hnorm : 1.f, &hexp);
  const float hscale = ldexpf(1.f, -hexp);  // exact: eigenvalues scale back by 2^hexp
  qr_bar();
  for (int idx = tid; idx < n * n; idx += 32 * QR_WARPS) {
    const int i = idx % n, j = idx / n;
    if (i <= j + 1) HF(H, ldh, i, j) *= hscale;
  }
  hnorm *= hscale;
  qr_bar();
  int hi = n - 1, steps = 0, since = 0;
  const int cap = 40 * n;
  while (hi >= 0) {
    // deflation (Algorithm 7.5.2): the largest lo <= hi with a negligible
    // H(lo, lo-1), which is set to zero; candidates tested 32 at a time
    int lo = 0;
    for (int top = hi; top > 0; top -= 32) {
      const int cand = top - lane;
      bool small = false;
      if (cand > 0) {
        float d = fabsf(HF(H, ldh, cand - 1, cand - 1)) + fabsf(HF(H, ldh, cand, cand));
        if (d == 0.f) d = hnorm;
        small = fabsf(HF(H, ldh, cand, cand - 1)) <= ulp * d;
      }
      const unsigned hits = __ballot_sync(0xffffffffu, small);
      if (hits) {
        lo = top - (__ffs(hits) - 1);
        break;
      }
    }
    qr_bar();
    if (lo > 0 && tid == 0) HF(H, ldh, lo, lo - 1) = 0.f;
    qr_bar();
    if (lo == hi) {  // a 1 x 1 block
      if (tid == 0) {
        wr[hi] = ldexpf(HF(H, ldh, hi, hi), hexp);
        wi[hi] = 0.f;
      }
      hi -= 1;
      since = 0;
      continue;
    }
    if (lo == hi - 1) {  // a 2 x 2 block
      if (tid == 0) {
        eig2x2(HF(H, ldh, hi - 1, hi - 1), HF(H, ldh, hi - 1, hi), HF(H, ldh, hi, hi - 1), HF(H, ldh, hi, hi),
               wr[hi - 1], wi[hi - 1], wr[hi], wi[hi]);
        wr[hi - 1] = ldexpf(wr[hi - 1], hexp);
        wi[hi - 1] = ldexpf(wi[hi - 1], hexp);
        wr[hi] = ldexpf(wr[hi], hexp);
        wi[hi] = ldexpf(wi[hi], hexp);
      }
      hi -= 2;
      since = 0;
      continue;
    }
    if (steps >= cap) {
      for (int i = tid; i <= hi; i += 32 * QR_WARPS) {
        wr[i] = NAN;
        wi[i] = 0.f;
      }
      qr_bar();
      return false;
    }
    ++steps;
    ++since;
    // the double shift: trace and determinant of the trailing 2 x 2 block; an
    // ad hoc real shift after every ten steps without deflation
    float tr, dt;
    if (since % 10 == 0) {
      const float g = HF(H, ldh, hi, hi) + 1.5f * (fabsf(HF(H, ldh, hi, hi - 1)) + fabsf(HF(H, ldh, hi - 1, hi - 2)));
      tr = 2.f * g;
      dt = g * g;
    } else {
      const float p = HF(H, ldh, hi - 1, hi - 1), q = HF(H, ldh, hi - 1, hi);
      const float r = HF(H, ldh, hi, hi - 1), s = HF(H, ldh, hi, hi);
      tr = p + s;
      dt = p * s - q * r;
    }
    // where the bulge starts, and the first column (x, y, z) of
    // (H - s1 I)(H - s2 I) from there (Algorithm 7.5.1): the largest m with a
    // negligible |H(m, m-1)| (|y| + |z|) against |x| times the neighbouring
    // diagonal, or lo; candidates tested 32 at a time
    int m0 = lo;
    float x = 0.f, y = 0.f, z = 0.f;
    for (int top = hi - 2; top >= lo; top -= 32) {
      const int cand = top - lane;
      bool stop = false;
      float cx = 0.f, cy = 0.f, cz = 0.f;
      if (cand >= lo) {
        const float g00 = HF(H, ldh, cand, cand), g01 = HF(H, ldh, cand, cand + 1);
        const float g10 = HF(H, ldh, cand + 1, cand), g11 = HF(H, ldh, cand + 1, cand + 1);
        cx = g00 * g00 + g01 * g10 - tr * g00 + dt;
        cy = g10 * (g00 + g11 - tr);
        cz = g10 * HF(H, ldh, cand + 2, cand + 1);
        stop = cand == lo || fabsf(HF(H, ldh, cand, cand - 1)) * (fabsf(cy) + fabsf(cz)) <=
                                 ulp * fabsf(cx) * (fabsf(HF(H, ldh, cand - 1, cand - 1)) + fabsf(g00) + fabsf(g11));
      }
      const unsigned hits = __ballot_sync(0xffffffffu, stop);
      if (hits) {
        const int src = __ffs(hits) - 1;
        m0 = top - src;
        x = __shfl_sync(0xffffffffu, cx, src);
        y = __shfl_sync(0xffffffffu, cy, src);
        z = __shfl_sync(0xffffffffu, cz, src);
        break;
      }
    }
    // bulge chase: the reflector of step a acts on indices a, a+1 (, a+2); a
    // start m0 > lo also transforms column m0 - 1, whose fill below the
    // subdiagonal is the negligible part dropped with the zeroing below
    for (int a = m0; a <= hi - 1; ++a) {
      const bool three = a + 2 <= hi;
      const Refl P = house3(x, y, three ? z : 0.f);
      const int q = a > lo ? a - 1 : lo;      // first column of the row transformation
      const int near = a + 3 < hi ? a + 3 : hi;  // last column near the bulge, last row of the column transformation
      float nx = 0.f, ny = 0.f, nz = 0.f;
      if (P.beta != 0.f) {
        if (wrp == 0) {
          // rows a..a+2 on columns q..near, then columns a..a+2 on rows a..near:
          // each lane takes one column, then one row; lane-parallel within the warp
          if (lane <= near - q) {
            const int j = q + lane;
            const float r0 = HF(H, ldh, a, j), r1 = HF(H, ldh, a + 1, j), r2 = three ? HF(H, ldh, a + 2, j) : 0.f;
            const float w = P.beta * (r0 + P.v1 * r1 + P.v2 * r2);
            HF(H, ldh, a, j) = r0 - w;
            HF(H, ldh, a + 1, j) = r1 - w * P.v1;
            if (three) HF(H, ldh, a + 2, j) = r2 - w * P.v2;
          }
          __syncwarp();
          if (lane <= near - a) {
            const int i = a + lane;
            const float c0 = HF(H, ldh, i, a), c1 = HF(H, ldh, i, a + 1), c2 = three ? HF(H, ldh, i, a + 2) : 0.f;
            const float w = P.beta * (c0 + P.v1 * c1 + P.v2 * c2);
            HF(H, ldh, i, a) = c0 - w;
            HF(H, ldh, i, a + 1) = c1 - w * P.v1;
            if (three) HF(H, ldh, i, a + 2) = c2 - w * P.v2;
          }
          __syncwarp();
          if (lane == 0) {
            if (a > lo) {  // the bulge column below the subdiagonal is now zero
              HF(H, ldh, a + 1, a - 1) = 0.f;
              if (three) HF(H, ldh, a + 2, a - 1) = 0.f;
            }
            if (a + 1 <= hi - 1) {  // the next reflector's input: column a of rows a+1..a+3
              nx = HF(H, ldh, a + 1, a);
              ny = HF(H, ldh, a + 2, a);
              nz = a + 3 <= hi ? HF(H, ldh, a + 3, a) : 0.f;
            }
          }
        } else if (wrp <= QR_RW) {
          const int off = 32 * (wrp - 1) + lane, stride = 32 * QR_RW;
          if (hi - (near + 1) < 2 * stride) {
            refl_rows<2>(H, ldh, a, three, P, near + 1, hi, off, stride);
          } else {
            refl_rows<(D_MAX + 32 * QR_RW - 1) / (32 * QR_RW)>(H, ldh, a, three, P, near + 1, hi, off, stride);
          }
        } else {
          const int off = 32 * (wrp - 1 - QR_RW) + lane, stride = 32 * QR_CW;
          if (a - 1 - lo < 2 * stride) {
            refl_cols<2>(H, ldh, a, three, P, lo, a - 1, off, stride);
          } else {
            refl_cols<(D_MAX + 32 * QR_CW - 1) / (32 * QR_CW)>(H, ldh, a, three, P, lo, a - 1, off, stride);
          }
        }
      } else if (wrp == 0 && lane == 0 && a + 1 <= hi - 1) {
        nx = HF(H, ldh, a + 1, a);
        ny = HF(H, ldh, a + 2, a);
        nz = a + 3 <= hi ? HF(H, ldh, a + 3, a) : 0.f;
      }
      float* slot = sh + 4 * (a & 1);  // alternating slots: one barrier per step suffices
      if (tid == 0) {
        slot[0] = nx;
        slot[1] = ny;
        slot[2] = nz;
      }
      qr_bar();
      x = slot[0];
      y = slot[1];
      z = slot[2];
    }
  }
  return true;
}

__global__ void __launch_bounds__(512, 1) k_ce_eig(WS ws) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  CeLayout L = ce_layout(ws.dscr);
  if (n <= 0) {  // SAW of numerical rank 0 (e.g. a breakdown on the first column): no candidates
    if (threadIdx.x == 0) L.cnt[0] = 0;
    return;
  }
  extern __shared__ float shf[];
  const int ldh = n + 1;
  float* H = shf;                 // n x n, ld n+1
  float* wr = H + ldh * n;        // n
  float* wi = wr + n;             // n
  float* red = wi + n;            // 32
  __shared__ float tau_s;
  __shared__ int ok;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n;
    HF(H, ldh, i, jj) = (float)L.M[i + (int64_t)jj * LDD];
  }
  __syncthreads();
  // --- Householder reduction to Hessenberg form (FP32) ---
  for (int col = 0; col + 2 < n; ++col) {
    float xs = 0.f;
    for (int i = col + 2 + threadIdx.x; i < n; i += blockDim.x) xs += HF(H, ldh, i, col) * HF(H, ldh, i, col);
    xs = block_sum_f(xs, red);
    if (xs == 0.f) {  // already reduced: the identity (tau = 0, a zero reflector below)
      if (threadIdx.x == 0) L.tauH[col] = 0.0;
      continue;
    }
    const float alpha = HF(H, ldh, col + 1, col);
    const float beta = -copysignf(sqrtf(alpha * alpha + xs), alpha);
    const float tau = (beta - alpha) / beta;
    const float sc = 1.f / (alpha - beta);
    for (int i = col + 2 + threadIdx.x; i < n; i += blockDim.x) HF(H, ldh, i, col) *= sc;
    if (threadIdx.x == 0) {
      HF(H, ldh, col + 1, col) = beta;
      tau_s = tau;
      L.tauH[col] = (double)tau;
    }
    __syncthreads();
    // left: four threads per column jj >= col+1, each a quarter of the rows
    // (interleaved), the dot reduced over the four lanes by shuffles
    for (int base = 4 * (col + 1); base < 4 * n; base += blockDim.x) {
      const int g = base + threadIdx.x, jj = g >> 2, sub = g & 3;
      const bool on = jj < n;
      float w = 0.f;
      const float h1 = on ? HF(H, ldh, col + 1, jj) : 0.f;  // read before the shuffles: sub 0 writes it after
      if (on)
        for (int i = col + 2 + sub; i < n; i += 4) w += HF(H, ldh, i, col) * HF(H, ldh, i, jj);
      w += __shfl_xor_sync(0xffffffffu, w, 1);
      w += __shfl_xor_sync(0xffffffffu, w, 2);
      if (on) {
        w = (w + h1) * tau_s;
        if (sub == 0) HF(H, ldh, col + 1, jj) -= w;
        for (int i = col + 2 + sub; i < n; i += 4) HF(H, ldh, i, jj) -= w * HF(H, ldh, i, col);
      }
    }
    __syncthreads();
    // right: four threads per row i, each a quarter of the columns (interleaved)
    for (int base = 0; base < 4 * n; base += blockDim.x) {
      const int g = base + threadIdx.x, i = g >> 2, sub = g & 3;
      const bool on = i < n;
      float w = 0.f;
      const float h1 = on ? HF(H, ldh, i, col + 1) : 0.f;  // read before the shuffles: sub 0 writes it after
      if (on)
        for (int jj = col + 2 + sub; jj < n; jj += 4) w += HF(H, ldh, i, jj) * HF(H, ldh, jj, col);
      w += __shfl_xor_sync(0xffffffffu, w, 1);
      w += __shfl_xor_sync(0xffffffffu, w, 2);
      if (on) {
        w = (w + h1) * tau_s;
        if (sub == 0) HF(H, ldh, i, col + 1) -= w;
        for (int jj = col + 2 + sub; jj < n; jj += 4) HF(H, ldh, i, jj) -= w * HF(H, ldh, jj, col);
      }
    }
    __syncthreads();
  }
  // the Hessenberg form with its reflectors (v = (1, H(col+2:n, col)), tau) for the
  // eigenvector starts of k_ce_invit
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n;
    L.H32[i + (int64_t)jj * LDD] = HF(H, ldh, i, jj);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n;
    if (i > jj + 1) HF(H, ldh, i, jj) = 0.f;
  }
  __syncthreads();
  __shared__ float rsl[8];
  if (threadIdx.x < 32 * QR_WARPS) {
    const bool good = francis_eigenvalues(H, ldh, n, wr, wi, rsl);
    if (threadIdx.x == 0) ok = good ? 1 : 0;
  }
  __syncthreads();
  // --- candidates: k + KC_MARGIN largest |mu| (FP32 order), pairs whole ---
  // The order: larger |mu| first, then larger real part, then lower index (a
  // strict total order); each thread ranks its eigenvalues against all others.
  // (a value the iteration left as NaN sorts last, so the ranks stay a permutation)
  __shared__ float mag[D_MAX], wrs[D_MAX];
  __shared__ int ord[D_MAX];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float h = hypotf(wr[i], wi[i]);
    mag[i] = isnan(h) ? -1.f : h;
    wrs[i] = isnan(wr[i]) ? -INFINITY : wr[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float mi = mag[i], ri = wrs[i];
    int rank = 0;
    for (int j2 = 0; j2 < n; ++j2) {
      const float mj = mag[j2], rj = wrs[j2];
      rank += (mj > mi) || (mj == mi && rj > ri) || (mj == mi && rj == ri && j2 < i);
    }
    ord[rank] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!ok) c->rankfail = 1;
    int kc = ws.k + KC_MARGIN < n ? ws.k + KC_MARGIN : n;
    if (kc > 0 && kc < n) {
      const int a = ord[kc - 1], b = ord[kc];
      if (wi[a] != 0.f && wr[b] == wr[a] && wi[b] == -wi[a]) kc += 1;
    }
    int nc = 0;
    for (int q = 0; q < kc && nc < KC; ++q) {
      const int e = ord[q];
      if (wi[e] < 0.f) continue;  // its conjugate partner (wi > 0) stands for the pair
      L.cmu[2 * nc] = wr[e];
      L.cmu[2 * nc + 1] = wi[e];
      ++nc;
    }
    L.cnt[0] = nc;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    L.wr[i] = wr[i];
    L.wi[i] = wi[i];
  }
}

size_t ce_eig_smem() { return ((size_t)(D_MAX + 1) * D_MAX + 2 * D_MAX + 64) * sizeof(float); }

// ---------------------------------------------------------------------------
// FP64 eigenpair of M for one candidate mu0 (one CTA each), with every
// dependent chain in FP32 and only independent row products in FP64 (a
// full-warp FP64 instruction holds an SM sub-partition for tens of cycles on
// this GPU, so a scalar FP64 chain, as in an FP64 LU, is slow):
//  1. inverse iteration from x = (1, ..., 1) on the FP32 Hessenberg form
//     H = Q^T fp32(M) Q that k_ce_eig computed (an O(n^2) LU of H - mu0 I),
//     IV_STEPS solves, then x0 = Q y to FP32 accuracy;
//  2. x0 scaled to x0(s) = 1 at an entry s of largest magnitude, and lambda0
//     the FP64 Rayleigh quotient x0^H M x0 / x0^H x0;
//  3. the refinement of Dongarra, Moler and Wilkinson (Improving the accuracy
//     of computed eigenvalues and eigenvectors, SIAM J. Numer. Anal. 20,
//     1983): Newton's method for (M - lambda I) x = 0 with x(s) = 1, whose
//     Jacobian is M - lambda I with column s replaced by -x, frozen at
//     (lambda0, x0) and factored once in FP32.  Each step computes the FP64
//     residual r = lambda x - M x, solves B z = r with the FP32 factors and
//     sets x(i) += z(i) (i != s), lambda += z(s); the FP64 residual carries
//     the accuracy.  The pair with the smallest max |r| seen is kept; if
//     its residual is not at the FP64 level (slow or no contraction, which
//     happens when M is too ill-conditioned for FP32 factors), the
//     candidate is flagged for the FP64 fallback below.
// M is scaled by a power of two 2^-e (exact) before rounding to FP32.
// ---------------------------------------------------------------------------
constexpr int IV_T = 512;
static_assert(IV_T >= D_MAX && IV_T % 32 == 0, "the solves give each row of M its own thread");
constexpr int IV_STEPS = 2;   // inverse-iteration solves before the refinement
constexpr int DMW_STEPS = 3;  // refinement steps
constexpr int IV_NQ = (D_MAX + 31) / 32;  // rows per lane in the LU update

struct cf {
  float re, im;
};
__device__ __forceinline__ cf cf_mul(cf a, cf b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// 1 / d in FP32 (d scaled to a largest component of one first); 0 for d = 0.
// The hardware reciprocal (within 2 ulp) suffices: these factors only
// precondition the FP64 refinement.
__device__ __forceinline__ cf cf_recip(cf d) {
  const float m = fmaxf(fabsf(d.re), fabsf(d.im));
  if (!(m > 0.f) || !isfinite(m)) return {0.f, 0.f};
  const float im = __fdividef(1.f, m);
  const float a = d.re * im, b = d.im * im;
  const float r = __fdividef(im, a * a + b * b);
  return {a * r, -b * r};
}

struct IvShared {
  float pr, pi, ir, ii;  // pivot value and its reciprocal
  int p;
};

// In-place FP32 LU with partial pivoting (pivot by |re| + |im|, ties the
// lowest row) of the n x n matrix (Ar, Ai), column-major with leading
// dimension ld, in shared memory: unit lower L below the diagonal, U on and
// above it, rows exchanged across the whole matrix (L included) and perm[k]
// the row exchanged with row k at step k.  A zero pivot is replaced by tiny.
// Kept out of line (as is iv_solve): inlined into k_ce_invit, whose FP64
// values stay live across it, the loops below picked up FP64 instructions
// (about 30,000 per factorisation, measured), each holding a sub-partition's
// FP64 pipe for tens of cycles; out of line the factorisation runs without
// them and takes 0.25 ms instead of 0.40 ms at n = 121.
// Block-wide, two or three barriers per step.  Warp 0 stores the previous
// step's multipliers (its registers) and pivot, and finds the pivot of column
// k; every warp forms the multipliers of its lanes' rows i = k + 1 + lane +
// 32 q from column k; the block exchanges rows k and p; then warp w updates
// its columns j = w (mod nw) one by one, over the row strips below k only.
__device__ __noinline__ void iv_lu(float* Ar, float* Ai, int ld, int n, bool cx, int* perm, float tiny, IvShared& sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  cf l[IV_NQ];
#pragma unroll
  for (int q = 0; q < IV_NQ; ++q) l[q] = cf{0.f, 0.f};
  for (int k = 0; k < n; ++k) {
    if (wid == 0) {
      if (k > 0) {  // the multipliers and the pivot of step k - 1 into column k - 1
#pragma unroll
        for (int q = 0; q < IV_NQ; ++q) {
          if (k + 32 * q >= n) break;  // uniform
          const int i = k + lane + 32 * q;
          if (i < n) {
            Ar[i + (k - 1) * ld] = l[q].re;
            if (cx) Ai[i + (k - 1) * ld] = l[q].im;
          }
        }
        if (lane == 0) {
          Ar[(k - 1) + (k - 1) * ld] = sh.pr;
          if (cx) Ai[(k - 1) + (k - 1) * ld] = sh.pi;
        }
        __syncwarp();
      }
      float best = -1.f;
      int bi = k;
#pragma unroll
      for (int q = 0; q < IV_NQ; ++q) {
        const int i = k + lane + 32 * q;
        if (i < n) {
          const float a = fabsf(Ar[i + k * ld]) + (cx ? fabsf(Ai[i + k * ld]) : 0.f);
          if (a > best) {
            best = a;
            bi = i;
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        cf pv{Ar[bi + k * ld], cx ? Ai[bi + k * ld] : 0.f};
        if (pv.re == 0.f && pv.im == 0.f) pv.re = tiny;
        const cf iv = cf_recip(pv);
        perm[k] = bi;
        sh.p = bi;
        sh.pr = pv.re;
        sh.pi = pv.im;
        sh.ir = iv.re;
        sh.ii = iv.im;
      }
    }
    __syncthreads();
    const int p = sh.p;
    const cf inv{sh.ir, sh.ii};
    // multipliers of this lane's rows from column k (row p holds the old row k's entry)
#pragma unroll
    for (int q = 0; q < IV_NQ; ++q) {
      if (k + 1 + 32 * q >= n) break;  // uniform
      const int i = k + 1 + lane + 32 * q;
      if (i < n) {
        const int src = i == p ? k : i;
        l[q] = cf_mul(cf{Ar[src + k * ld], cx ? Ai[src + k * ld] : 0.f}, inv);
      } else {
        l[q] = cf{0.f, 0.f};
      }
    }
    // row exchange, one thread per column (consecutive columns, an odd ld: no bank
    // conflicts), then the update
    if (p != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (j == k) continue;
        float t = Ar[k + j * ld];
        Ar[k + j * ld] = Ar[p + j * ld];
        Ar[p + j * ld] = t;
        if (cx) {
          t = Ai[k + j * ld];
          Ai[k + j * ld] = Ai[p + j * ld];
          Ai[p + j * ld] = t;
        }
      }
      __syncthreads();
    }
    int j = wid;
    while (j <= k) j += nw;  // this warp's first column right of k
    for (; j < n; j += nw) {
      const float ur = Ar[k + j * ld], ui = cx ? Ai[k + j * ld] : 0.f;
#pragma unroll
      for (int q = 0; q < IV_NQ; ++q) {
        if (k + 1 + 32 * q >= n) break;  // the strips below row k only (uniform)
        const int i = k + 1 + lane + 32 * q;
        if (i < n) {
          if (cx) {
            const float ar = Ar[i + j * ld], ai = Ai[i + j * ld];
            Ar[i + j * ld] = ar - (l[q].re * ur - l[q].im * ui);
            Ai[i + j * ld] = ai - (l[q].re * ui + l[q].im * ur);
          } else {
            Ar[i + j * ld] = fmaf(-l[q].re, ur, Ar[i + j * ld]);
          }
        }
      }
    }
    __syncthreads();
  }
  // the last step's pivot (no multipliers below it)
  if (threadIdx.x == 0) {
    Ar[(n - 1) + (n - 1) * ld] = sh.pr;
    if (cx) Ai[(n - 1) + (n - 1) * ld] = sh.pi;
  }
  __syncthreads();
}

// Row k of P y is y[sig[k]]: the exchanges of the factorisation composed.
__device__ void iv_perm(const int* perm, int n, int* sig) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < n; ++k) sig[k] = k;
    for (int k = 0; k < n; ++k) {
      const int p = perm[k];
      const int t = sig[k];
      sig[k] = sig[p];
      sig[p] = t;
    }
  }
}

// Solve L U y = (yr, yi) in place (y already permuted; out of line, as iv_lu) with the first
// nb = 32 ceil(n / 32) threads: thread t owns row t and loads the next
// column's factor entry of its row ahead of time; the value of column k
// passes through shared memory (alternating slots) with one named barrier of
// those threads per column.  (udr, udi): reciprocals of U's diagonal; slot:
// 8 floats of shared memory.
__device__ __noinline__ void iv_solve(const float* Ar, const float* Ai, int ld, int n, bool cx, float* yr, float* yi,
                         const float* udr, const float* udi, float* slot) {
  const int t = threadIdx.x;
  const int nb = (n + 31) & ~31;
  if (t >= nb) return;
  const bool own = t < n;
  float vr = own ? yr[t] : 0.f, vi = (own && cx) ? yi[t] : 0.f;
  // L y = b: at column k, y_k is final; rows t > k subtract L(t, k) y_k
  float fr = (own && t > 0) ? Ar[t] : 0.f, fi = (own && t > 0 && cx) ? Ai[t] : 0.f;
  for (int k = 0; k < n; ++k) {
    const bool nx = own && t > k + 1;
    const float gr = nx ? Ar[t + (k + 1) * ld] : 0.f, gi = (nx && cx) ? Ai[t + (k + 1) * ld] : 0.f;
    float* sl = slot + 2 * (k & 1);
    if (t == k) {
      sl[0] = vr;
      sl[1] = vi;
    }
    asm volatile("bar.sync 2, %0;" ::"r"(nb) : "memory");
    const float yk_r = sl[0], yk_i = sl[1];
    if (cx) {
      vr -= fr * yk_r - fi * yk_i;
      vi -= fr * yk_i + fi * yk_r;
    } else {
      vr = fmaf(-fr, yk_r, vr);
    }
    fr = gr;
    fi = gi;
  }
  // U x = y: x_k = y_k / U(k, k), then rows t < k subtract U(t, k) x_k (its
  // own pair of slots, so that no write races a read of the last L column)
  slot += 4;
  fr = (own && t < n - 1) ? Ar[t + (n - 1) * ld] : 0.f;
  fi = (own && t < n - 1 && cx) ? Ai[t + (n - 1) * ld] : 0.f;
  for (int k = n - 1; k >= 0; --k) {
    const bool nx = own && k >= 1 && t < k - 1;
    const float gr = nx ? Ar[t + (k - 1) * ld] : 0.f, gi = (nx && cx) ? Ai[t + (k - 1) * ld] : 0.f;
    float* sl = slot + 2 * (k & 1);
    if (t == k) {
      const float xr = cx ? vr * udr[k] - vi * udi[k] : vr * udr[k];
      const float xi = cx ? vr * udi[k] + vi * udr[k] : 0.f;
      vr = xr;
      vi = xi;
      sl[0] = xr;
      sl[1] = xi;
    }
    asm volatile("bar.sync 2, %0;" ::"r"(nb) : "memory");
    const float xk_r = sl[0], xk_i = sl[1];
    if (cx) {
      vr -= fr * xk_r - fi * xk_i;
      vi -= fr * xk_i + fi * xk_r;
    } else {
      vr = fmaf(-fr, xk_r, vr);
    }
    fr = gr;
    fi = gi;
  }
  if (own) {
    yr[t] = vr;
    if (cx) yi[t] = vi;
  }
}

// (M x)_i for a row i of M (global, column-major, ld LDD) and x = xr + i xi in
// shared memory; the loads of M run eight columns ahead of the FMAs.
__device__ __forceinline__ void iv_row_dot(const double* __restrict__ M, int n, int i, const double* xr,
                                           const double* xi, double& sr, double& si) {
  constexpr int G = 8;
  sr = 0.0;
  si = 0.0;
  const double* __restrict__ row = M + i;
  int j = 0;
  for (; j + G <= n; j += G) {
    double mv[G];
#pragma unroll
    for (int u = 0; u < G; ++u) mv[u] = __ldg(row + (int64_t)(j + u) * LDD);
#pragma unroll
    for (int u = 0; u < G; ++u) {
      sr = fma(mv[u], xr[j + u], sr);
      si = fma(mv[u], xi[j + u], si);
    }
  }
  for (; j < n; ++j) {
    const double m = __ldg(row + (int64_t)j * LDD);
    sr = fma(m, xr[j], sr);
    si = fma(m, xi[j], si);
  }
}

// (rr, ri) = lambda x - M x in FP64; returns max_i max(|re r_i|, |im r_i|) to
// every thread.
__device__ double iv_residual(const double* __restrict__ M, int n, double lr, double li, const double* xr,
                              const double* xi, double* rr, double* ri, unsigned long long* redu) {
  unsigned long long mb = 0ull;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double sr, si;
    iv_row_dot(M, n, i, xr, xi, sr, si);
    const double a = fma(lr, xr[i], fma(-li, xi[i], -sr));
    const double b = fma(lr, xi[i], fma(li, xr[i], -si));
    rr[i] = a;
    ri[i] = b;
    const unsigned long long u = abs_bits(a), v = abs_bits(b);
    const unsigned long long w = u > v ? u : v;
    mb = w > mb ? w : mb;
  }
  mb = block_max_u64(mb, redu);
  return __longlong_as_double((long long)mb);
}

// 2^(1022 - e) for a biased exponent e of a positive value v: v 2^(1022 - e)
// lies in [0.5, 1).  1 when e is out of the range where that is a normal double.
__device__ __forceinline__ double iv_pow2_scale(int e) {
  return e >= 1 && e <= 2043 ? __longlong_as_double((long long)((unsigned long long)(2045 - e) << 52)) : 1.0;
}

size_t ce_invit_smem() {
  return (size_t)2 * D_MAX * (D_MAX + 1) * sizeof(float) + 4 * D_MAX * sizeof(float) +
         6 * D_MAX * sizeof(double) + 2 * D_MAX * sizeof(int);
}

__global__ void __launch_bounds__(IV_T, 1) k_ce_invit(WS ws) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  CeLayout L = ce_layout(ws.dscr);
  const int idx = blockIdx.x;
  if (n <= 0 || idx >= L.cnt[0]) return;
  if (c->svd_path) {  // the truncated problem: M is ill-conditioned, FP32 factors do not contract;
    if (threadIdx.x == 0) L.ivfail[idx] = 1;  // the FP64 inverse iteration takes every candidate
    return;
  }
  extern __shared__ __align__(16) unsigned char iv_smem[];
  double* xr = (double*)iv_smem;  // the eigenvector (FP64)
  double* xi = xr + D_MAX;
  double* rr = xi + D_MAX;        // residual
  double* ri = rr + D_MAX;
  double* br = ri + D_MAX;        // the best pair so far
  double* bi = br + D_MAX;
  float* yr = (float*)(bi + D_MAX);  // FP32 solve vector
  float* yi = yr + D_MAX;
  float* udr = yi + D_MAX;           // reciprocals of U's diagonal
  float* udi = udr + D_MAX;
  int* perm = (int*)(udi + D_MAX);
  int* sig = perm + D_MAX;
  const int ld = n | 1;  // odd: a row walk across columns hits every bank once
  float* Ar = (float*)(sig + D_MAX);
  float* Ai = Ar + (size_t)ld * n;
  __shared__ IvShared sh;
  __shared__ float iv_slot[8];
  __shared__ unsigned long long redu[32];
  __shared__ double red[32];
  __shared__ double lam_s[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* __restrict__ M = L.M;
  const double mu_r = L.cmu[2 * idx], mu_i = L.cmu[2 * idx + 1];
  // Complex candidate: Im mu0 != 0, tested on its bits (no FP64 instruction).
  const bool cx = ((unsigned long long)__double_as_longlong(mu_i) << 1) != 0ull;
  // the power-of-two scale of M (loads of a column issued together)
  unsigned long long mb = 0ull;
  for (int j = wid; j < n; j += nw) {
    double v[IV_NQ];
#pragma unroll
    for (int q = 0; q < IV_NQ; ++q) {
      const int i = lane + 32 * q;
      v[q] = i < n ? __ldg(M + i + (int64_t)j * LDD) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < IV_NQ; ++q) {
      const unsigned long long u = abs_bits(v[q]);
      mb = u > mb ? u : mb;
    }
  }
  mb = block_max_u64(mb, redu);
  const double sc = iv_pow2_scale(bexp_of_bits(mb));  // max |M sc| in [0.5, 1)
  const float tiny = 5.9604645e-8f * (float)n;         // 2^-24 n, against entries of order one
  // ---- 1. x0: inverse iteration on the FP32 Hessenberg form H = Q^T fp32(M) Q that
  // k_ce_eig left in L.H32, then x0 = Q y.  The LU of H - mu0 I (pivoting between
  // rows k and k + 1) is O(n^2); U stays in (Ar, Ai) with zeros below the diagonal,
  // the multipliers in (rr, ri) and the exchanges in perm. ----
  for (int j = wid; j < n; j += nw) {
#pragma unroll
    for (int q = 0; q < IV_NQ; ++q) {
      const int i = lane + 32 * q;
      if (i < n) {
        const float h = i <= j + 1 ? L.H32[i + (int64_t)j * LDD] : 0.f;
        Ar[i + j * ld] = i == j ? h - (float)mu_r : h;
        if (cx) Ai[i + j * ld] = i == j ? (float)(-mu_i) : 0.f;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    float hmax = 0.f;  // the largest diagonal magnitude, for the zero-pivot replacement
    for (int e = lane; e < n; e += 32) hmax = fmaxf(hmax, fabsf(Ar[e + e * ld]));
    for (int o = 16; o > 0; o >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    const float htiny = fmaxf(hmax, 1e-30f) * 5.9604645e-8f * (float)n;
    for (int k = 0; k + 1 < n; ++k) {
      const cf a0{Ar[k + k * ld], cx ? Ai[k + k * ld] : 0.f};
      const cf a1{Ar[k + 1 + k * ld], cx ? Ai[k + 1 + k * ld] : 0.f};
      const bool sw = fabsf(a1.re) + fabsf(a1.im) > fabsf(a0.re) + fabsf(a0.im);
      __syncwarp();
      if (sw)
        for (int j = k + lane; j < n; j += 32) {
          float t = Ar[k + j * ld];
          Ar[k + j * ld] = Ar[k + 1 + j * ld];
          Ar[k + 1 + j * ld] = t;
          if (cx) {
            t = Ai[k + j * ld];
            Ai[k + j * ld] = Ai[k + 1 + j * ld];
            Ai[k + 1 + j * ld] = t;
          }
        }
      __syncwarp();
      cf pv = sw ? a1 : a0;
      if (pv.re == 0.f && pv.im == 0.f) pv.re = htiny;
      const cf l = cf_mul(sw ? a0 : a1, cf_recip(pv));
      for (int j = k + 1 + lane; j < n; j += 32) {
        const cf u{Ar[k + j * ld], cx ? Ai[k + j * ld] : 0.f};
        Ar[k + 1 + j * ld] -= l.re * u.re - l.im * u.im;
        if (cx) Ai[k + 1 + j * ld] -= l.re * u.im + l.im * u.re;
      }
      if (lane == 0) {
        Ar[k + k * ld] = pv.re;
        if (cx) Ai[k + k * ld] = pv.im;
        Ar[k + 1 + k * ld] = 0.f;
        if (cx) Ai[k + 1 + k * ld] = 0.f;
        rr[k] = (double)l.re;
        ri[k] = (double)l.im;
        perm[k] = sw ? 1 : 0;
      }
      __syncwarp();
    }
    if (lane == 0 && Ar[(n - 1) + (n - 1) * ld] == 0.f && (!cx || Ai[(n - 1) + (n - 1) * ld] == 0.f))
      Ar[(n - 1) + (n - 1) * ld] = htiny;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const cf r = cf_recip(cf{Ar[k + k * ld], cx ? Ai[k + k * ld] : 0.f});
    udr[k] = r.re;
    udi[k] = r.im;
    yr[k] = 1.f;
    yi[k] = 0.f;
  }
  __syncthreads();
  for (int it = 0; it < IV_STEPS; ++it) {
    // P L (exchanges and multipliers, in order), then U (iv_solve: its L pass finds
    // zeros), then the scale to a largest |re| + |im| of one
    if (threadIdx.x == 0) {
      for (int k = 0; k + 1 < n; ++k) {
        cf y0{yr[k], yi[k]}, y1{yr[k + 1], yi[k + 1]};
        if (perm[k]) {
          const cf t = y0;
          y0 = y1;
          y1 = t;
        }
        const cf l{(float)rr[k], (float)ri[k]};
        const cf ly = cf_mul(l, y0);
        yr[k] = y0.re;
        yi[k] = y0.im;
        yr[k + 1] = y1.re - ly.re;
        yi[k + 1] = cx ? y1.im - ly.im : 0.f;
      }
    }
    __syncthreads();
    iv_solve(Ar, Ai, ld, n, cx, yr, yi, udr, udi, iv_slot);
    __syncthreads();
    if (threadIdx.x < 32) {
      float best = -1.f;
      int bix = 0;
      for (int i = lane; i < n; i += 32) {
        const float a = fabsf(yr[i]) + fabsf(yi[i]);
        if (a > best) {
          best = a;
          bix = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bix, o);
        if (ob > best || (ob == best && oi < bix)) {
          best = ob;
          bix = oi;
        }
      }
      const cf inv = best > 0.f && isfinite(best) ? cf_recip(cf{yr[bix], yi[bix]}) : cf{1.f, 0.f};
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        const cf v = cf_mul(cf{yr[i], yi[i]}, inv);
        yr[i] = v.re;
        yi[i] = cx ? v.im : 0.f;
      }
    }
    __syncthreads();
  }
  // x0 = Q y: the reflectors (staged in Ar) applied in reverse order, by warp 0
  for (int j = wid; j + 2 < n; j += nw)
    for (int i = j + 2 + lane; i < n; i += 32) Ar[i + j * ld] = L.H32[i + (int64_t)j * LDD];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int col = n - 3; col >= 0; --col) {
      const float tau = (float)L.tauH[col];
      if (tau == 0.f) continue;  // uniform
      float dr = 0.f, di = 0.f;
      for (int i = col + 1 + lane; i < n; i += 32) {
        const float v = i == col + 1 ? 1.f : Ar[i + col * ld];
        dr = fmaf(v, yr[i], dr);
        di = fmaf(v, yi[i], di);
      }
      for (int o = 16; o > 0; o >>= 1) {
        dr += __shfl_xor_sync(0xffffffffu, dr, o);
        di += __shfl_xor_sync(0xffffffffu, di, o);
      }
      __syncwarp();
      for (int i = col + 1 + lane; i < n; i += 32) {
        const float v = i == col + 1 ? 1.f : Ar[i + col * ld];
        yr[i] = fmaf(-tau * dr, v, yr[i]);
        if (cx) yi[i] = fmaf(-tau * di, v, yi[i]);
      }
      __syncwarp();
    }
    // the entry of largest |re| + |im| (x0(s) = 1 below)
    float best = -1.f;
    int bix = 0;
    for (int i = lane; i < n; i += 32) {
      const float a = fabsf(yr[i]) + fabsf(yi[i]);
      if (a > best) {
        best = a;
        bix = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bix, o);
      if (ob > best || (ob == best && oi < bix)) {
        best = ob;
        bix = oi;
      }
    }
    const cf inv = best > 0.f && isfinite(best) ? cf_recip(cf{yr[bix], yi[bix]}) : cf{1.f, 0.f};
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      const cf v = cf_mul(cf{yr[i], yi[i]}, inv);
      yr[i] = v.re;
      yi[i] = cx ? v.im : 0.f;
    }
    if (lane == 0) sh.p = bix;
  }
  __syncthreads();
  // ---- 2. x0 with x0(s) = 1, lambda0 = Rayleigh quotient ----
  const int s = sh.p;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    xr[i] = i == s ? 1.0 : (double)yr[i];
    xi[i] = (i == s || !cx) ? 0.0 : (double)yi[i];
  }
  __syncthreads();
  {
    double nr = 0.0, ni = 0.0, dd = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double sr, si;
      iv_row_dot(M, n, i, xr, xi, sr, si);
      nr += xr[i] * sr + xi[i] * si;  // conj(x_i) (M x)_i
      ni += xr[i] * si - xi[i] * sr;
      dd += xr[i] * xr[i] + xi[i] * xi[i];
    }
    nr = block_sum(nr, red);
    ni = block_sum(ni, red);
    dd = block_sum(dd, red);
    if (threadIdx.x == 0) {
      lam_s[0] = nr / dd;
      lam_s[1] = cx ? ni / dd : 0.0;
    }
    __syncthreads();
  }
  double lr = lam_s[0], li = lam_s[1];
  // ---- 3. B = (M - lambda0 I) sc with column s replaced by -x0 sc, in FP32 ----
  for (int j = wid; j < n; j += nw) {
    double v[IV_NQ];
#pragma unroll
    for (int q = 0; q < IV_NQ; ++q) {
      const int i = lane + 32 * q;
      v[q] = (i < n && j != s) ? __ldg(M + i + (int64_t)j * LDD) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < IV_NQ; ++q) {
      const int i = lane + 32 * q;
      if (i >= n) continue;
      if (j == s) {
        Ar[i + j * ld] = (float)(-xr[i] * sc);
        if (cx) Ai[i + j * ld] = (float)(-xi[i] * sc);
      } else {
        Ar[i + j * ld] = (float)(i == j ? (v[q] - lr) * sc : v[q] * sc);
        if (cx) Ai[i + j * ld] = i == j ? (float)(-li * sc) : 0.f;
      }
    }
  }
  __syncthreads();
  iv_lu(Ar, Ai, ld, n, cx, perm, tiny, sh);
  iv_perm(perm, n, sig);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const cf r = cf_recip(cf{Ar[k + k * ld], cx ? Ai[k + k * ld] : 0.f});
    udr[k] = r.re;
    udi[k] = r.im;
  }
  __syncthreads();
  double best = INFINITY;
  double blr = lr, bli = li;  // the pair kept when no residual is finite: x0, lambda0
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    br[i] = xr[i];
    bi[i] = xi[i];
  }
  for (int it = 0; it <= DMW_STEPS; ++it) {
    const double rmax = iv_residual(M, n, lr, li, xr, xi, rr, ri, redu);
    if (rmax < best) {  // uniform: every thread holds the same rmax
      best = rmax;
      blr = lr;
      bli = li;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        br[i] = xr[i];
        bi[i] = xi[i];
      }
    }
    if (it == DMW_STEPS || !(rmax > 0.0) || !isfinite(rmax)) break;
    // B z = r, with r scaled by a power of two to a largest entry of order one
    const double rs = iv_pow2_scale(bexp_of_bits((unsigned long long)__double_as_longlong(rmax)));
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      yr[i] = (float)(rr[sig[i]] * rs);
      yi[i] = cx ? (float)(ri[sig[i]] * rs) : 0.f;
    }
    __syncthreads();
    iv_solve(Ar, Ai, ld, n, cx, yr, yi, udr, udi, iv_slot);
    __syncthreads();
    // z = y sc / rs (B was scaled by sc, r by rs)
    const double zs = sc / rs;
    const double dlr = (double)yr[s] * zs, dli = cx ? (double)yi[s] * zs : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (i == s) continue;
      xr[i] += (double)yr[i] * zs;
      if (cx) xi[i] += (double)yi[i] * zs;
    }
    lr += dlr;
    li += dli;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    L.cref[2 * idx] = blr;
    L.cref[2 * idx + 1] = cx ? bli : 0.0;
    // converged: the best residual at the level of its own FP64 rounding (n eps max|M| max|x|,
    // with max|x| about one), with a margin of 256; else the FP64 fallback takes the candidate
    const double mmax = __longlong_as_double((long long)mb);
    L.ivfail[idx] = (best <= 256.0 * (double)n * 2.220446049250313e-16 * mmax) ? 0 : 1;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    L.cvec[i + (int64_t)(2 * idx) * LDD] = br[i];
    L.cvec[i + (int64_t)(2 * idx + 1) * LDD] = bi[i];
  }
}

// ---------------------------------------------------------------------------
// The fallback for a candidate whose refinement above did not reach FP64
// accuracy (flagged in ivfail): FP64 eigenpair of M by LU with partial
// pivoting of M - mu0 I (complex when Im mu0 != 0), three steps of inverse
// iteration, and the Rayleigh quotient mu = x^H M x / x^H x.  One CTA per
// candidate; the others return at once.  Slow on this GPU (its pivot chain
// is FP64), but its accuracy does not depend on the conditioning of M, which
// the FP32 factors of the refinement do: on the truncated-SVD path M can be
// too ill-conditioned for them.
// ---------------------------------------------------------------------------
struct cplx { double re, im; };
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
// 1 / d for a complex d: conj(d) / |d|^2 with |d|^2 scaled into range by a
// power of two and its reciprocal from an FP32 estimate refined by two Newton
// steps r <- r (2 - q r) (an FP64 division is a long instruction sequence on
// this GPU; these are a few dependent FMAs).
__device__ inline cplx crecip(cplx d) {
  const double m = fmax(fabs(d.re), fabs(d.im));
  if (!(m > 0.0) || !isfinite(m)) return cplx{0.0, 0.0};
  const int e = (int)(((unsigned long long)__double_as_longlong(m) >> 52) & 0x7FF) - 1023;
  const int ec = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
  const double sc = __longlong_as_double((long long)((unsigned long long)(1023 - ec) << 52));  // 2^-ec
  const double ar = d.re * sc, ai = d.im * sc;          // |scaled| in [1, 2)
  const double q = fma(ar, ar, ai * ai);                 // in [1, 8)
  double r = (double)__frcp_rn((float)q);
  r = r * fma(-q, r, 2.0);
  r = r * fma(-q, r, 2.0);
  r = r * fma(-q, r, 2.0);
  // 1/d = conj(d_s) / q * sc
  return cplx{ar * r * sc, -ai * r * sc};
}


__global__ void __launch_bounds__(512) k_ce_invit64(WS ws) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  CeLayout L = ce_layout(ws.dscr);
  const int idx = blockIdx.x;
  if (n <= 0 || idx >= L.cnt[0] || !L.ivfail[idx]) return;
  const cplx mu0{L.cmu[2 * idx], L.cmu[2 * idx + 1]};
  const bool cx = mu0.im != 0.0;
  double* Ar = L.lu + (int64_t)idx * 2 * LDD * LDD;  // column-major n x n
  double* Ai = Ar + (int64_t)LDD * LDD;
  __shared__ double xr[D_MAX], xi[D_MAX];
  __shared__ int perm[D_MAX];
  __shared__ double red[32];
  __shared__ double bc[4];
  __shared__ unsigned long long redu[32];
  const double* M = L.M;
  double mnorm = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    const double v = M[i + (int64_t)j * LDD];
    Ar[i + (int64_t)j * LDD] = v - (i == j ? mu0.re : 0.0);
    Ai[i + (int64_t)j * LDD] = (i == j) ? -mu0.im : 0.0;
    mnorm = fmax(mnorm, fabs(v));
  }
  {  // block max via the u64 bit pattern of a non-negative double
    unsigned long long b = (unsigned long long)__double_as_longlong(mnorm);
    b = block_max_u64(b, redu);
    mnorm = __longlong_as_double((long long)b);
  }
  const double tiny = fmax(mnorm, 1e-300) * 2.220446049250313e-16 * (double)n;
  __syncthreads();
  // LU with partial pivoting (pivot by |re| + |im|)
  for (int k = 0; k < n; ++k) {
    unsigned long long best = 0ull;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const double a = fabs(Ar[i + (int64_t)k * LDD]) + (cx ? fabs(Ai[i + (int64_t)k * LDD]) : 0.0);
      // pack (magnitude bits, row) so that the max picks the largest, ties the lowest row
      const unsigned long long key = ((unsigned long long)__double_as_longlong(a) & ~0x3FFull) |
                                     (unsigned long long)(0x3FF - i);
      best = key > best ? key : best;
    }
    best = block_max_u64(best, redu);
    const int p = 0x3FF - (int)(best & 0x3FF);
    if (threadIdx.x == 0) perm[k] = p;
    if (p != k) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double t = Ar[k + (int64_t)j * LDD];
        Ar[k + (int64_t)j * LDD] = Ar[p + (int64_t)j * LDD];
        Ar[p + (int64_t)j * LDD] = t;
        if (cx) {
          t = Ai[k + (int64_t)j * LDD];
          Ai[k + (int64_t)j * LDD] = Ai[p + (int64_t)j * LDD];
          Ai[p + (int64_t)j * LDD] = t;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      cplx d{Ar[k + (int64_t)k * LDD], cx ? Ai[k + (int64_t)k * LDD] : 0.0};
      if (d.re == 0.0 && d.im == 0.0) {
        d.re = tiny;
        Ar[k + (int64_t)k * LDD] = tiny;
      }
      const cplx inv = crecip(d);
      bc[0] = inv.re;
      bc[1] = inv.im;
    }
    __syncthreads();
    const cplx inv{bc[0], bc[1]};
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      if (cx) {
        const cplx l = cmul(cplx{Ar[i + (int64_t)k * LDD], Ai[i + (int64_t)k * LDD]}, inv);
        Ar[i + (int64_t)k * LDD] = l.re;
        Ai[i + (int64_t)k * LDD] = l.im;
      } else {
        Ar[i + (int64_t)k * LDD] *= inv.re;
      }
    }
    __syncthreads();
    const int m = n - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e % m, j = k + 1 + e / m;
      if (cx) {
        const cplx l{Ar[i + (int64_t)k * LDD], Ai[i + (int64_t)k * LDD]};
        const cplx u{Ar[k + (int64_t)j * LDD], Ai[k + (int64_t)j * LDD]};
        const cplx a = csub(cplx{Ar[i + (int64_t)j * LDD], Ai[i + (int64_t)j * LDD]}, cmul(l, u));
        Ar[i + (int64_t)j * LDD] = a.re;
        Ai[i + (int64_t)j * LDD] = a.im;
      } else {
        Ar[i + (int64_t)j * LDD] = fma(-Ar[i + (int64_t)k * LDD], Ar[k + (int64_t)j * LDD], Ar[i + (int64_t)j * LDD]);
      }
    }
    __syncthreads();
  }
  // inverse iteration from x = (1, ..., 1); the reciprocals of U's diagonal
  // are formed once, in parallel, so the back substitution only multiplies
  __shared__ double udr[D_MAX], udi[D_MAX];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const cplx inv = crecip(cplx{Ar[k + (int64_t)k * LDD], cx ? Ai[k + (int64_t)k * LDD] : 0.0});
    udr[k] = inv.re;
    udi[k] = inv.im;
  }
  // the row interchanges of the factorisation as one permutation: row k of
  // P x is x[sig[k]]
  __shared__ int sig[D_MAX];
  __shared__ double yr[D_MAX], yi[D_MAX];
  if (threadIdx.x == 0) {
    for (int k = 0; k < n; ++k) sig[k] = k;
    for (int k = 0; k < n; ++k) {
      const int p = perm[k];
      const int t = sig[k];
      sig[k] = sig[p];
      sig[p] = t;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) { xr[i] = 1.0; xi[i] = 0.0; }
  __syncthreads();
  // The triangular solves: thread t owns row t (n <= D_MAX <= blockDim.x)
  // and keeps the next PF entries of its row of L (or U) in flight, so the
  // L2 latency of the factors stays off the column-by-column chain; one
  // barrier of the first nb threads per column.
  constexpr int PF = 4;
  const int t = threadIdx.x;
  const bool own = t < n;
  const int nb = (n + 31) / 32 * 32;
  const bool inb = t < nb;
  for (int it = 0; it < 3; ++it) {
    if (own) {
      yr[t] = xr[sig[t]];
      yi[t] = xi[sig[t]];
    }
    __syncthreads();
    if (inb) {
      // L y = P x (unit lower): at column k, rows t > k take y_k
      cplx lp[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u)
        lp[u] = (own && u < t) ? cplx{Ar[t + (int64_t)u * LDD], cx ? Ai[t + (int64_t)u * LDD] : 0.0} : cplx{0.0, 0.0};
      for (int k0 = 0; k0 < n; k0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
          const int k = k0 + u;
          if (k < n) {
            if (own && t > k) {
              const cplx v = csub(cplx{yr[t], yi[t]}, cmul(lp[u], cplx{yr[k], yi[k]}));
              yr[t] = v.re;
              yi[t] = v.im;
            }
            const int kn = k + PF;
            lp[u] = (own && kn < t) ? cplx{Ar[t + (int64_t)kn * LDD], cx ? Ai[t + (int64_t)kn * LDD] : 0.0}
                                    : cplx{0.0, 0.0};
            asm volatile("bar.sync 2, %0;" ::"r"(nb) : "memory");
          }
        }
      }
      // U x = y (upper), columns from the last: x_k = y_k / u_kk, then rows t < k
      cplx up[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int kk = n - 1 - u;
        up[u] = (own && kk > t) ? cplx{Ar[t + (int64_t)kk * LDD], cx ? Ai[t + (int64_t)kk * LDD] : 0.0}
                                : cplx{0.0, 0.0};
      }
      for (int k0 = n - 1; k0 >= 0; k0 -= PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
          const int k = k0 - u;
          if (k >= 0) {
            const cplx xk = cmul(cplx{yr[k], yi[k]}, cplx{udr[k], udi[k]});
            if (own && t < k) {
              const cplx v = csub(cplx{yr[t], yi[t]}, cmul(up[u], xk));
              yr[t] = v.re;
              yi[t] = v.im;
            }
            if (t == k) {
              xr[k] = xk.re;
              xi[k] = xk.im;
            }
            const int kn = k - PF;
            up[u] = (own && kn > t && kn >= 0)
                        ? cplx{Ar[t + (int64_t)kn * LDD], cx ? Ai[t + (int64_t)kn * LDD] : 0.0}
                        : cplx{0.0, 0.0};
            asm volatile("bar.sync 2, %0;" ::"r"(nb) : "memory");
          }
        }
      }
    }
    __syncthreads();
    // normalise by the entry of largest |re| + |im| (ties: lowest index)
    unsigned long long key = 0ull;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double a = fabs(xr[i]) + fabs(xi[i]);
      const unsigned long long kk =
          ((unsigned long long)__double_as_longlong(a) & ~0x3FFull) | (unsigned long long)(0x3FF - i);
      key = kk > key ? kk : key;
    }
    key = block_max_u64(key, redu);
    const int bi = 0x3FF - (int)(key & 0x3FF);
    const cplx piv{xr[bi], xi[bi]};
    const cplx inv = (piv.re == 0.0 && piv.im == 0.0) ? cplx{1.0, 0.0} : crecip(piv);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const cplx v = cmul(cplx{xr[i], xi[i]}, inv);
      xr[i] = v.re;
      xi[i] = cx ? v.im : 0.0;
    }
    __syncthreads();
  }
  // Rayleigh quotient mu = x^H M x / x^H x
  double nr = 0.0, ni = 0.0, dd = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double yr = 0.0, yi = 0.0;
    for (int j = 0; j < n; ++j) {
      const double mij = M[i + (int64_t)j * LDD];
      yr = fma(mij, xr[j], yr);
      yi = fma(mij, xi[j], yi);
    }
    // conj(x_i) * y_i
    nr += xr[i] * yr + xi[i] * yi;
    ni += xr[i] * yi - xi[i] * yr;
    dd += xr[i] * xr[i] + xi[i] * xi[i];
  }
  nr = block_sum(nr, red);
  ni = block_sum(ni, red);
  dd = block_sum(dd, red);
  if (threadIdx.x == 0) {
    L.cref[2 * idx] = nr / dd;
    L.cref[2 * idx + 1] = cx ? ni / dd : 0.0;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    L.cvec[i + (int64_t)(2 * idx) * LDD] = xr[i];
    L.cvec[i + (int64_t)(2 * idx + 1) * LDD] = xi[i];
  }
}

// Selection on the FP64 eigenvalues: the k largest |mu| (ties: larger real
// part, lower candidate index); a pair counts twice and is kept whole.
__global__ void k_ce_select(WS ws) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  CeLayout L = ce_layout(ws.dscr);
  __shared__ int ord[KC];
  __shared__ int zc_of[KC];
  __shared__ int nsel;
  const int nc = n > 0 ? L.cnt[0] : 0;  // rank 0: nothing to select, no recycle columns
  if (threadIdx.x == 0) {
    for (int i = 0; i < nc; ++i) ord[i] = i;
    for (int i = 1; i < nc; ++i) {
      const int v = ord[i];
      const double mv = hypot(L.cref[2 * v], L.cref[2 * v + 1]);
      int y = i - 1;
      while (y >= 0) {
        const int u = ord[y];
        const double mu = hypot(L.cref[2 * u], L.cref[2 * u + 1]);
        const bool after = (mu < mv) || (mu == mv && L.cref[2 * u] < L.cref[2 * v]) ||
                           (mu == mv && L.cref[2 * u] == L.cref[2 * v] && u > v);
        if (!after) break;
        ord[y + 1] = u;
        --y;
      }
      ord[y + 1] = v;
    }
    int cols = 0, q = 0;
    while (q < nc && cols < ws.k) {
      const int e = ord[q];
      zc_of[q] = cols;
      cols += (L.cref[2 * e + 1] != 0.0) ? 2 : 1;
      ++q;
    }
    if (cols > K_MAX) cols = K_MAX;
    nsel = q;
    c->kprime = cols;
  }
  __syncthreads();
  for (int q = 0; q < nsel; ++q) {
    const int e = ord[q];
    const int zc = zc_of[q];
    const bool cx = L.cref[2 * e + 1] != 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      L.Zr[i + (int64_t)zc * LDD] = L.cvec[i + (int64_t)(2 * e) * LDD];
      if (cx && zc + 1 < K_MAX) L.Zr[i + (int64_t)(zc + 1) * LDD] = L.cvec[i + (int64_t)(2 * e + 1) * LDD];
    }
  }
}

// ---------------------------------------------------------------------------
// Orthonormal basis Z of the selected eigenvectors (MGS, two passes), P, the
// alpha-scaled P' for the tall update, and the cycle log.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_ce_finish(WS ws, int kh, int ucur) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  const int d = kh + c->jf;
  const int kp = c->kprime;
  CeLayout L = ce_layout(ws.dscr);
  __shared__ double red[32];
  __shared__ double dts[K_MAX];
  int zdep = 0;  // (thread 0) a selected eigenvector depends on the earlier ones
  double* Z = L.Zr;
  for (int col = 0; col < kp; ++col) {
    double* zc = Z + (int64_t)col * LDD;
    double n0 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) n0 = fma(zc[i], zc[i], n0);
    n0 = sqrt(block_sum(n0, red));
    // classical Gram-Schmidt, twice (as stable as modified Gram-Schmidt twice);
    // all projections of a pass at once, one warp per earlier column
    for (int pass = 0; pass < 2; ++pass) {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int q = wid; q < col; q += nw) {
        const double* zq = Z + (int64_t)q * LDD;
        double dt = 0.0;
        for (int i = lane; i < n; i += 32) dt = fma(zq[i], zc[i], dt);
        dt = warp_sum(dt);
        if (lane == 0) dts[q] = dt;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = zc[i];
        for (int q = 0; q < col; ++q) v = fma(-dts[q], Z[i + (int64_t)q * LDD], v);
        zc[i] = v;
      }
      __syncthreads();
    }
    double nr = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) nr = fma(zc[i], zc[i], nr);
    nr = sqrt(block_sum(nr, red));
    if (threadIdx.x == 0 && !(nr > 1e-12 * n0)) {
      c->rankfail = 1;
      zdep = 1;
    }
    const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) zc[i] *= inv;
    __syncthreads();
  }
  // P = V_l Z (truncated-SVD path) or Z (full-rank path); P' scales V rows by alpha
  const bool svd = c->svd_path != 0;
  for (int idx = threadIdx.x; idx < d * K_MAX; idx += blockDim.x) {
    const int l = idx % d, col = idx / d;
    double v = 0.0;
    if (col < kp) {
      if (svd) {
        for (int q = 0; q < n; ++q) v = fma(L.Vh[l + (int64_t)q * LDD], Z[q + (int64_t)col * LDD], v);
      } else {
        v = Z[l + (int64_t)col * LDD];
      }
    }
    L.Pu[l + (int64_t)col * LDD] = v;
    ws.P[l + (int64_t)col * D_MAX] = l < kh ? v : v * c->alpha[l - kh];
  }
  __syncthreads();
  // fixed-point P'' = diag(2^(E_l)) P' per column for the tall update, where
  // 2^(-E_l) scales column l of [U V] to a maximum in [0.5, 1)
  {
    __shared__ unsigned long long redu[32];
    for (int col = 0; col < kp; ++col) {
      unsigned long long mb = 0ull;
      for (int l = threadIdx.x; l < d; l += blockDim.x) {
        const unsigned long long cb = l < kh ? c->umax[ucur][l] : c->vmax[l - kh];
        const int ce = bexp_of_bits(cb);
        const double pv = ws.P[l + (int64_t)col * D_MAX];
        const double pp = ce == 0 ? 0.0 : ldexp(pv, ce - 1022);
        L.Hc[l] = pp;  // scratch row (Hc is unused here)
        const unsigned long long u = abs_bits(pp);
        mb = u > mb ? u : mb;
      }
      mb = block_max_u64(mb, redu);
      const int emax = bexp_of_bits(mb);
      for (int l = threadIdx.x; l < d; l += blockDim.x) {
        const Q52 q = q52(L.Hc[l], emax, 0);
        ws.Pq[l + (int64_t)col * D_MAX] = ((unsigned long long)(unsigned)q.hi << 32) | (unsigned long long)q.lo;
      }
      if (threadIdx.x == 0) ws.Pexp[col] = emax - 1022;
      __syncthreads();
    }
    for (int col = threadIdx.x; col < K_MAX; col += blockDim.x) c->umax[1 - ucur][col] = 0ull;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int li = c->log_n;
    if (li < LOG_MAX) {
      CycleLog g;
      g.steps = c->jf;
      g.checks = c->nchecks;
      g.converged = c->converged;
      g.ell = c->ell;
      g.kprime = kp;
      g.kh = kh;
      g.flags = (c->svd_path ? 1 : 0) | (c->breakdown ? 2 : 0) | (c->rankfail ? 4 : 0) | (zdep ? 8 : 0);
      g.svd_sweeps = c->svd_path ? c->svd_sweeps : 0;
      g.res = c->res;
      g.sres = c->sres;
      g.safety = c->safety;
      ws.log[li] = g;
    }
    c->log_n = li + 1;
  }
}

// SU_new(:, col) = S[U V] P(:, col), SAU_new(:, col) = SAW P(:, col).
__global__ void k_ce_sketch_update(WS ws, int kh, const double* __restrict__ SU, const double* __restrict__ SAU,
                                   double* __restrict__ SUn, double* __restrict__ SAUn) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int d = kh + c->jf;
  const int col = blockIdx.x;
  if (col >= c->kprime) return;
  CeLayout L = ce_layout(ws.dscr);
  __shared__ double pc[D_MAX];
  for (int l = threadIdx.x; l < d; l += blockDim.x) pc[l] = L.Pu[l + (int64_t)col * LDD];
  __syncthreads();
  for (int i = threadIdx.x; i < ws.s; i += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int l = 0; l < d; ++l) {
      a = fma(sv_col(ws, SU, kh, l)[i], pc[l], a);
      b = fma(saw_col(ws, SAU, kh, l)[i], pc[l], b);
    }
    SUn[i + (int64_t)col * ws.s] = a;
    SAUn[i + (int64_t)col * ws.s] = b;
  }
}

cudaError_t launch_cycle_end_part(int part, const WS& ws, int kh, int ucur, const double* SU, const double* SAU,
                                  double* SUn, double* SAUn, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ce_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ce_eig_smem());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ce_invit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ce_invit_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int dmax_now = kh + ws.m;
  switch (part) {
    case 0: k_ce_formC<<<dmax_now, 256, 0, st>>>(ws, SU, kh); break;
    case 1: k_ce_rinv<<<dmax_now, 32, 0, st>>>(ws, kh); break;
    case 2: k_ce_M<<<dmax_now, 256, 0, st>>>(ws, kh); break;
    case 3: {
      static bool attr_done = false;
      if (!attr_done) {
        const cudaError_t ea = cudaFuncSetAttribute(k_ce_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)ce_svd_smem());
        if (ea != cudaSuccess) return ea;
        attr_done = true;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(SVD_CTAS, 1, 1);
      cfg.blockDim = dim3(512, 1, 1);
      cfg.dynamicSmemBytes = ce_svd_smem();
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = SVD_CTAS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, k_ce_svd, ws, kh);
      if (e != cudaSuccess) return e;
      break;
    }
    case 4: k_ce_eig<<<1, 512, ce_eig_smem(), st>>>(ws); break;
    case 5:
      k_ce_invit<<<KC, IV_T, ce_invit_smem(), st>>>(ws);
      k_ce_invit64<<<KC, 512, 0, st>>>(ws);  // the candidates the refinement left, if any
      break;
    case 6: k_ce_select<<<1, 256, 0, st>>>(ws); break;
    case 7: k_ce_finish<<<1, 512, 0, st>>>(ws, kh, ucur); break;
    case 8: k_ce_sketch_update<<<K_MAX, 512, 0, st>>>(ws, kh, SU, SAU, SUn, SAUn); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sdr
