// Cycle end of GMRES-SDR: sketched harmonic-Ritz update of the recycle space
// (Section 3.4 and the last block of Algorithm 1), FP64.
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
// Eigenpairs: Householder reduction to Hessenberg form, Francis double-shift
// QR for the eigenvalues, inverse iteration with the Hessenberg matrix for the
// selected eigenvectors, back-transformation, and an orthonormal real basis of
// their span (real and imaginary parts of complex pairs).
#include "launch.cuh"

namespace sdr {

constexpr int LDD = D_MAX;  // leading dimension of the d x d scratch matrices

struct CeLayout {
  double *C, *Rinv, *M, *Hc, *Vh, *As, *tauH, *wr, *wi, *Zr, *Pu, *colsq, *misc, *lu;
  int* sel;   // [K_MAX] eigenvalue index per inverse iteration
  int* zcol;  // [K_MAX] first Z column of that eigenvalue
  int* cnt;   // [0] number of inverse iterations
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
  L.lu = L.misc + 64 + 3 * K_MAX;  // K_MAX blocks of 2*LDD*LDD (complex LU)
  return L;
}

size_t ce_scratch_doubles() { return (size_t)6 * LDD * LDD + 3 * LDD + 2 * (size_t)LDD * K_MAX + 2 * LDD + 64 +
                                     3 * K_MAX + (size_t)K_MAX * 2 * LDD * LDD + 64; }

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
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_ce_svd(WS ws, int kh) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0 || !c->svd_path) return;
  const int d = kh + c->jf;
  CeLayout L = ce_layout(ws.dscr);
  double* A = L.As;   // working matrix (d x d)
  double* V = L.Vh;   // right singular vectors
  __shared__ double sig[D_MAX];
  __shared__ int order[D_MAX];
  __shared__ int rotated;
  const int ld = ws.dmax;
  for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) {
    const int i = idx % d, jj = idx / d;
    A[i + (int64_t)jj * LDD] = i <= jj ? ws.Rf[i + (int64_t)jj * ld] : 0.0;
    V[i + (int64_t)jj * LDD] = (i == jj) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int dd = d + (d & 1);  // even number of players; index d (if odd) is a dummy
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double eps = 2.220446049250313e-16;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < dd - 1; ++round) {
      for (int k = wid; k < dd / 2; k += nw) {
        int a, b;
        if (k == 0) {
          a = 0;
          b = 1 + (round % (dd - 1));
        } else {
          a = 1 + ((k + round) % (dd - 1));
          b = 1 + ((dd - 1 - k + round) % (dd - 1));
        }
        if (a > b) { int tmp = a; a = b; b = tmp; }
        if (b >= d) continue;
        double* ap = A + (int64_t)a * LDD;
        double* aq = A + (int64_t)b * LDD;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < d; i += 32) {
          al = fma(ap[i], ap[i], al);
          be = fma(aq[i], aq[i], be);
          ga = fma(ap[i], aq[i], ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (!(fabs(ga) > eps * sqrt(al * be)) || al == 0.0 || be == 0.0) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        double* vp = V + (int64_t)a * LDD;
        double* vq = V + (int64_t)b * LDD;
        for (int i = lane; i < d; i += 32) {
          const double x1 = ap[i], x2 = aq[i];
          ap[i] = cs * x1 - sn * x2;
          aq[i] = sn * x1 + cs * x2;
          const double y1 = vp[i], y2 = vq[i];
          vp[i] = cs * y1 - sn * y2;
          vq[i] = sn * y1 + cs * y2;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  // singular values and ordering (descending)
  for (int i = wid; i < d; i += nw) {
    double a = 0.0;
    for (int r = lane; r < d; r += 32) a = fma(A[r + (int64_t)i * LDD], A[r + (int64_t)i * LDD], a);
    a = warp_sum(a);
    if (lane == 0) sig[i] = sqrt(a);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < d; ++i) order[i] = i;
    for (int i = 1; i < d; ++i) {  // insertion sort, stable
      int v = order[i], y = i - 1;
      while (y >= 0 && sig[order[y]] < sig[v]) { order[y + 1] = order[y]; --y; }
      order[y + 1] = v;
    }
    const double s1 = sig[order[0]];
    int ell = 0;
    for (int i = 0; i < d; ++i) ell += sig[order[i]] > s1 * (double)d * eps ? 1 : 0;
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
    for (int l = 0; l < d; ++l) a = fma(L.C[i + (int64_t)l * LDD], vc[l], a);
    T1[i + (int64_t)q * LDD] = a;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ell * ell; idx += blockDim.x) {
    const int i = idx % ell, q = idx / ell;
    const double si = sig[order[i]];
    const double* uc = A + (int64_t)order[i] * LDD;
    double a = 0.0;
    for (int l = 0; l < d; ++l) a = fma(uc[l], T1[l + (int64_t)q * LDD], a);
    L.M[i + (int64_t)q * LDD] = a / (si * si);  // U_l = A_l / sigma, then S^{-1}
  }
  __syncthreads();
  // keep V_l (ordered) in the columns of As for P = V_l Z
  for (int idx = threadIdx.x; idx < d * ell; idx += blockDim.x) {
    const int i = idx % d, q = idx / d;
    T1[i + (int64_t)q * LDD] = V[i + (int64_t)order[q] * LDD];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < d * ell; idx += blockDim.x) {
    const int i = idx % d, q = idx / d;
    V[i + (int64_t)q * LDD] = T1[i + (int64_t)q * LDD];
  }
}

// ---------------------------------------------------------------------------
// Hessenberg reduction + Francis double-shift QR (eigenvalues) + selection.
// H lives in shared memory with leading dimension n+1.
// ---------------------------------------------------------------------------
__device__ inline double& HS(double* H, int ldh, int i, int j) { return H[i + j * ldh]; }

__global__ void __launch_bounds__(512) k_ce_eig(WS ws) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  if (n <= 0) return;
  CeLayout L = ce_layout(ws.dscr);
  extern __shared__ double shm[];
  const int ldh = n + 1;
  double* H = shm;                  // n x n, ld n+1
  double* tauH = H + ldh * n;       // n
  double* wr = tauH + n;            // n
  double* wi = wr + n;              // n
  double* red = wi + n;             // 32
  __shared__ int fail;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n;
    HS(H, ldh, i, jj) = L.M[i + (int64_t)jj * LDD];
  }
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // --- Householder reduction to upper Hessenberg form ---
  for (int col = 0; col + 2 < n; ++col) {
    double xs = 0.0;
    for (int i = col + 2 + threadIdx.x; i < n; i += blockDim.x) xs = fma(HS(H, ldh, i, col), HS(H, ldh, i, col), xs);
    xs = block_sum(xs, red);
    const double alpha = HS(H, ldh, col + 1, col);
    double tau = 0.0, beta = alpha, sc = 0.0;
    if (xs != 0.0) {
      beta = -copysign(sqrt(alpha * alpha + xs), alpha);
      tau = (beta - alpha) / beta;
      sc = 1.0 / (alpha - beta);
    }
    __syncthreads();
    for (int i = col + 2 + threadIdx.x; i < n; i += blockDim.x) HS(H, ldh, i, col) *= sc;
    if (threadIdx.x == 0) {
      HS(H, ldh, col + 1, col) = beta;
      tauH[col] = tau;
    }
    __syncthreads();
    if (tau == 0.0) continue;
    // left: rows col+1.., columns col+1..n-1 (warp per column)
    for (int jj = col + 1 + wid; jj < n; jj += nw) {
      double w = HS(H, ldh, col + 1, jj) * (lane == 0 ? 1.0 : 0.0);
      for (int i = col + 2 + lane; i < n; i += 32) w = fma(HS(H, ldh, i, col), HS(H, ldh, i, jj), w);
      w = warp_sum(w) * tau;
      if (lane == 0) HS(H, ldh, col + 1, jj) -= w;
      for (int i = col + 2 + lane; i < n; i += 32) HS(H, ldh, i, jj) = fma(-w, HS(H, ldh, i, col), HS(H, ldh, i, jj));
    }
    __syncthreads();
    // right: all rows, columns col+1..n-1 (warp per row)
    for (int i = wid; i < n; i += nw) {
      double w = lane == 0 ? HS(H, ldh, i, col + 1) : 0.0;
      for (int jj = col + 2 + lane; jj < n; jj += 32) w = fma(HS(H, ldh, i, jj), HS(H, ldh, jj, col), w);
      w = warp_sum(w) * tau;
      if (lane == 0) HS(H, ldh, i, col + 1) -= w;
      for (int jj = col + 2 + lane; jj < n; jj += 32) HS(H, ldh, i, jj) = fma(-w, HS(H, ldh, jj, col), HS(H, ldh, i, jj));
    }
    __syncthreads();
  }
  // save reflectors (below the subdiagonal) and a clean Hessenberg copy
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n;
    const double v = HS(H, ldh, i, jj);
    L.M[i + (int64_t)jj * LDD] = v;  // reflectors kept below the subdiagonal
    L.Hc[i + (int64_t)jj * LDD] = (i <= jj + 1) ? v : 0.0;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) L.tauH[i] = i + 2 < n ? tauH[i] : 0.0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx % n, jj = idx / n;
    if (i > jj + 1) HS(H, ldh, i, jj) = 0.0;
  }
  double an = 0.0;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) an += fabs(HS(H, ldh, idx % n, idx / n));
  an = block_sum(an, red);
  if (threadIdx.x == 0) L.misc[0] = an;
  // --- Francis double-shift QR, one warp ---
  if (wid == 0) {
    const double eps = 2.220446049250313e-16;
    int nn = n - 1;
    double tsh = 0.0;
    int total = 0;
    while (nn >= 0) {
      int its = 0;
      while (true) {
        int l = nn;
        while (l > 0) {
          double s = fabs(HS(H, ldh, l - 1, l - 1)) + fabs(HS(H, ldh, l, l));
          if (s == 0.0) s = an;
          if (fabs(HS(H, ldh, l, l - 1)) <= eps * s) break;
          --l;
        }
        __syncwarp();
        if (l > 0 && lane == 0) HS(H, ldh, l, l - 1) = 0.0;
        __syncwarp();
        double x = HS(H, ldh, nn, nn);
        if (l == nn) {
          if (lane == 0) { wr[nn] = x + tsh; wi[nn] = 0.0; }
          nn -= 1;
          break;
        }
        double y = HS(H, ldh, nn - 1, nn - 1);
        double w = HS(H, ldh, nn, nn - 1) * HS(H, ldh, nn - 1, nn);
        if (l == nn - 1) {
          const double p = 0.5 * (y - x), q = p * p + w;
          double z = sqrt(fabs(q));
          x += tsh;
          if (lane == 0) {
            if (q >= 0.0) {
              z = p + copysign(z, p);
              wr[nn - 1] = wr[nn] = x + z;
              if (z != 0.0) wr[nn] = x - w / z;
              wi[nn - 1] = wi[nn] = 0.0;
            } else {
              wr[nn - 1] = wr[nn] = x + p;
              wi[nn - 1] = z;
              wi[nn] = -z;
            }
          }
          nn -= 2;
          break;
        }
        if (its >= 60 || total >= 60 * n) {
          if (lane == 0) fail = 1;
          for (int i = lane; i <= nn; i += 32) { wr[i] = NAN; wi[i] = 0.0; }
          nn = -1;
          break;
        }
        if (its == 10 || its == 20) {  // exceptional shift
          tsh += x;
          __syncwarp();
          for (int i = lane; i <= nn; i += 32) HS(H, ldh, i, i) -= x;
          __syncwarp();
          const double s = fabs(HS(H, ldh, nn, nn - 1)) + fabs(HS(H, ldh, nn - 1, nn - 2));
          x = y = 0.75 * s;
          w = -0.4375 * s * s;
        }
        ++its;
        ++total;
        int m = nn - 2;
        double p = 0.0, q = 0.0, r = 0.0, z = 0.0;
        while (true) {
          z = HS(H, ldh, m, m);
          const double rr = x - z, ss = y - z;
          p = (rr * ss - w) / HS(H, ldh, m + 1, m) + HS(H, ldh, m, m + 1);
          q = HS(H, ldh, m + 1, m + 1) - z - rr - ss;
          r = HS(H, ldh, m + 2, m + 1);
          const double sc = fabs(p) + fabs(q) + fabs(r);
          p /= sc; q /= sc; r /= sc;
          if (m == l) break;
          const double u = fabs(HS(H, ldh, m, m - 1)) * (fabs(q) + fabs(r));
          const double v = fabs(p) * (fabs(HS(H, ldh, m - 1, m - 1)) + fabs(z) + fabs(HS(H, ldh, m + 1, m + 1)));
          if (u <= eps * v) break;
          --m;
        }
        __syncwarp();
        for (int i = m + 2 + lane; i <= nn; i += 32) {
          HS(H, ldh, i, i - 2) = 0.0;
          if (i != m + 2) HS(H, ldh, i, i - 3) = 0.0;
        }
        __syncwarp();
        for (int k = m; k <= nn - 1; ++k) {
          if (k != m) {
            p = HS(H, ldh, k, k - 1);
            q = HS(H, ldh, k + 1, k - 1);
            r = (k != nn - 1) ? HS(H, ldh, k + 2, k - 1) : 0.0;
            x = fabs(p) + fabs(q) + fabs(r);
            if (x != 0.0) { p /= x; q /= x; r /= x; }
          }
          const double s = copysign(sqrt(p * p + q * q + r * r), p);
          __syncwarp();
          if (s != 0.0) {
            if (lane == 0) {
              if (k == m) {
                if (l != m) HS(H, ldh, k, k - 1) = -HS(H, ldh, k, k - 1);
              } else {
                HS(H, ldh, k, k - 1) = -s * x;
              }
            }
            p += s;
            const double xx = p / s, yy = q / s, zz = r / s;
            const double qq = q / p, rq = r / p;
            __syncwarp();
            for (int jj = k + lane; jj <= nn; jj += 32) {
              double pp = HS(H, ldh, k, jj) + qq * HS(H, ldh, k + 1, jj);
              if (k != nn - 1) {
                pp += rq * HS(H, ldh, k + 2, jj);
                HS(H, ldh, k + 2, jj) -= pp * zz;
              }
              HS(H, ldh, k + 1, jj) -= pp * yy;
              HS(H, ldh, k, jj) -= pp * xx;
            }
            __syncwarp();
            const int imax = nn < k + 3 ? nn : k + 3;
            for (int i = l + lane; i <= imax; i += 32) {
              double pp = xx * HS(H, ldh, i, k) + yy * HS(H, ldh, i, k + 1);
              if (k != nn - 1) {
                pp += zz * HS(H, ldh, i, k + 2);
                HS(H, ldh, i, k + 2) -= pp * rq;
              }
              HS(H, ldh, i, k + 1) -= pp * qq;
              HS(H, ldh, i, k) -= pp;
            }
            __syncwarp();
          }
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    L.wr[i] = wr[i];
    L.wi[i] = wi[i];
  }
  __syncthreads();
  // --- selection: k largest |mu| (ties: larger real part, lower index); a
  // complex-conjugate pair split at the boundary is kept whole ---
  if (threadIdx.x == 0) {
    if (fail) c->rankfail = 1;
    int ord[D_MAX];
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 1; i < n; ++i) {
      const int v = ord[i];
      const double mv = hypot(wr[v], wi[v]);
      int y = i - 1;
      while (y >= 0) {
        const int u = ord[y];
        const double mu = hypot(wr[u], wi[u]);
        const bool after = (mu < mv) || (mu == mv && wr[u] < wr[v]) || (mu == mv && wr[u] == wr[v] && u > v);
        if (!after) break;
        ord[y + 1] = u;
        --y;
      }
      ord[y + 1] = v;
    }
    int kk = ws.k < n ? ws.k : n;
    if (kk > 0 && kk < n) {
      const int a = ord[kk - 1], b = ord[kk];
      if (wi[a] != 0.0 && wr[b] == wr[a] && wi[b] == -wi[a]) kk += 1;
    }
    if (kk > K_MAX) kk = K_MAX;
    int ninv = 0, zc = 0;
    for (int q = 0; q < kk; ++q) {
      const int e = ord[q];
      if (wi[e] == 0.0) {
        L.sel[ninv] = e; L.zcol[ninv] = zc; ++ninv; zc += 1;
      } else if (wi[e] > 0.0) {
        L.sel[ninv] = e; L.zcol[ninv] = zc; ++ninv; zc += 2;
      }
    }
    if (zc > K_MAX) zc = K_MAX;
    L.cnt[0] = ninv;
    c->kprime = zc;
  }
}

size_t ce_eig_smem() { return ((size_t)(D_MAX + 1) * D_MAX + 3 * D_MAX + 32) * sizeof(double); }

// ---------------------------------------------------------------------------
// Inverse iteration (H - mu I) x = b on the Hessenberg matrix, one CTA per
// selected eigenvalue, complex arithmetic; then x <- Q_H x.
// ---------------------------------------------------------------------------
struct cplx { double re, im; };
__device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ inline double cabs2(cplx a) { return hypot(a.re, a.im); }
__device__ inline cplx cdiv(cplx a, cplx b) {  // Smith's algorithm
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, den = b.re + b.im * r;
    return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  }
  const double r = b.re / b.im, den = b.re * r + b.im;
  return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}

__global__ void __launch_bounds__(256) k_ce_invit(WS ws) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  CeLayout L = ce_layout(ws.dscr);
  const int idx = blockIdx.x;
  if (n <= 0 || idx >= L.cnt[0]) return;
  const int e = L.sel[idx];
  const cplx mu{L.wr[e], L.wi[e]};
  const bool is_cplx = mu.im != 0.0;
  double* Ure = L.lu + (int64_t)idx * 2 * LDD * LDD;  // row-major U(i, j) at i*LDD + j
  double* Uim = Ure + (int64_t)LDD * LDD;
  __shared__ double crr[D_MAX], cri[D_MAX], nrr[D_MAX], nri[D_MAX];
  __shared__ double mlr[D_MAX], mli[D_MAX];
  __shared__ int swp[D_MAX];
  __shared__ double xr[D_MAX], xi[D_MAX];
  __shared__ double red[32];
  __shared__ double bc[4];
  const double tiny = fmax(L.misc[0], 1e-300) * 2.220446049250313e-16;
  const double* Hc = L.Hc;
  for (int jj = threadIdx.x; jj < n; jj += blockDim.x) {
    crr[jj] = Hc[0 + (int64_t)jj * LDD] - (jj == 0 ? mu.re : 0.0);
    cri[jj] = jj == 0 ? -mu.im : 0.0;
  }
  __syncthreads();
  for (int i = 0; i + 1 < n; ++i) {
    for (int jj = i + threadIdx.x; jj < n; jj += blockDim.x) {
      nrr[jj] = Hc[(i + 1) + (int64_t)jj * LDD] - (jj == i + 1 ? mu.re : 0.0);
      nri[jj] = jj == i + 1 ? -mu.im : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      cplx a{crr[i], cri[i]}, b{nrr[i], nri[i]};
      const int s = cabs2(b) > cabs2(a) ? 1 : 0;
      cplx piv = s ? b : a, oth = s ? a : b;
      if (piv.re == 0.0 && piv.im == 0.0) piv.re = tiny;
      const cplx ml = cdiv(oth, piv);
      swp[i] = s;
      mlr[i] = ml.re;
      mli[i] = ml.im;
      bc[0] = piv.re;
      bc[1] = piv.im;
    }
    __syncthreads();
    const int s = swp[i];
    const cplx ml{mlr[i], mli[i]};
    for (int jj = i + threadIdx.x; jj < n; jj += blockDim.x) {
      cplx a{crr[jj], cri[jj]}, b{nrr[jj], nri[jj]};
      cplx up = s ? b : a, lo = s ? a : b;
      if (jj == i) { up.re = bc[0]; up.im = bc[1]; }
      Ure[(int64_t)i * LDD + jj] = up.re;
      Uim[(int64_t)i * LDD + jj] = up.im;
      const cplx nv = csub(lo, cmul(ml, up));
      crr[jj] = nv.re;
      cri[jj] = nv.im;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double r = crr[n - 1], im = cri[n - 1];
    if (r == 0.0 && im == 0.0) r = tiny;
    Ure[(int64_t)(n - 1) * LDD + (n - 1)] = r;
    Uim[(int64_t)(n - 1) * LDD + (n - 1)] = im;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) { xr[i] = 1.0; xi[i] = 0.0; }
  __syncthreads();
  for (int iter = 0; iter < 3; ++iter) {
    if (threadIdx.x == 0) {  // forward elimination of the right-hand side
      for (int i = 0; i + 1 < n; ++i) {
        if (swp[i]) {
          double t = xr[i]; xr[i] = xr[i + 1]; xr[i + 1] = t;
          t = xi[i]; xi[i] = xi[i + 1]; xi[i + 1] = t;
        }
        const cplx v = csub(cplx{xr[i + 1], xi[i + 1]}, cmul(cplx{mlr[i], mli[i]}, cplx{xr[i], xi[i]}));
        xr[i + 1] = v.re;
        xi[i + 1] = v.im;
      }
    }
    __syncthreads();
    for (int i = n - 1; i >= 0; --i) {  // back substitution, column oriented
      if (threadIdx.x == 0) {
        cplx d{Ure[(int64_t)i * LDD + i], Uim[(int64_t)i * LDD + i]};
        if (d.re == 0.0 && d.im == 0.0) d.re = tiny;
        const cplx v = cdiv(cplx{xr[i], xi[i]}, d);
        xr[i] = v.re;
        xi[i] = v.im;
      }
      __syncthreads();
      const cplx xv{xr[i], xi[i]};
      for (int l = threadIdx.x; l < i; l += blockDim.x) {
        const cplx v = csub(cplx{xr[l], xi[l]}, cmul(cplx{Ure[(int64_t)l * LDD + i], Uim[(int64_t)l * LDD + i]}, xv));
        xr[l] = v.re;
        xi[l] = v.im;
      }
      __syncthreads();
    }
    // normalise by the largest modulus (deterministic: first index attaining it)
    if (threadIdx.x == 0) {
      double best = -1.0;
      int bi = 0;
      for (int i = 0; i < n; ++i) {
        const double a = hypot(xr[i], xi[i]);
        if (a > best) { best = a; bi = i; }
      }
      const cplx piv{xr[bi], xi[bi]};
      bc[0] = piv.re;
      bc[1] = piv.im;
    }
    __syncthreads();
    const cplx piv{bc[0], bc[1]};
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const cplx v = (piv.re == 0.0 && piv.im == 0.0) ? cplx{xr[i], xi[i]} : cdiv(cplx{xr[i], xi[i]}, piv);
      xr[i] = v.re;
      xi[i] = is_cplx ? v.im : 0.0;
    }
    __syncthreads();
  }
  // x <- Q_H x with Q_H = H_0 H_1 ... H_{n-3}: apply H_{n-3} first
  for (int col = n - 3; col >= 0; --col) {
    const double tau = L.tauH[col];
    if (tau == 0.0) continue;
    double dr = 0.0, di = 0.0;
    for (int i = col + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double v = (i == col + 1) ? 1.0 : L.M[i + (int64_t)col * LDD];
      dr = fma(v, xr[i], dr);
      di = fma(v, xi[i], di);
    }
    dr = block_sum(dr, red);
    di = block_sum(di, red);
    for (int i = col + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double v = (i == col + 1) ? 1.0 : L.M[i + (int64_t)col * LDD];
      xr[i] = fma(-tau * dr, v, xr[i]);
      xi[i] = fma(-tau * di, v, xi[i]);
    }
    __syncthreads();
  }
  const int zc = L.zcol[idx];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    L.Zr[i + (int64_t)zc * LDD] = xr[i];
    if (is_cplx && zc + 1 < K_MAX) L.Zr[i + (int64_t)(zc + 1) * LDD] = xi[i];
  }
}

// ---------------------------------------------------------------------------
// Orthonormal basis Z of the selected eigenvectors (MGS, two passes), P, the
// alpha-scaled P' for the tall update, and the cycle log.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_ce_finish(WS ws, int kh) {
  Ctl* c = ws.ctl;
  if (c->jf <= 0) return;
  const int n = c->ell;
  const int d = kh + c->jf;
  const int kp = c->kprime;
  CeLayout L = ce_layout(ws.dscr);
  __shared__ double red[32];
  double* Z = L.Zr;
  for (int col = 0; col < kp; ++col) {
    double* zc = Z + (int64_t)col * LDD;
    double n0 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) n0 = fma(zc[i], zc[i], n0);
    n0 = sqrt(block_sum(n0, red));
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = 0; q < col; ++q) {
        const double* zq = Z + (int64_t)q * LDD;
        double dt = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) dt = fma(zq[i], zc[i], dt);
        dt = block_sum(dt, red);
        for (int i = threadIdx.x; i < n; i += blockDim.x) zc[i] = fma(-dt, zq[i], zc[i]);
        __syncthreads();
      }
    }
    double nr = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) nr = fma(zc[i], zc[i], nr);
    nr = sqrt(block_sum(nr, red));
    if (threadIdx.x == 0 && !(nr > 1e-12 * n0)) c->rankfail = 1;
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
      g.flags = (c->svd_path ? 1 : 0) | (c->breakdown ? 2 : 0) | (c->rankfail ? 4 : 0);
      g.pad = 0;
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

cudaError_t launch_cycle_end(const WS& ws, int kh, const double* SU, const double* SAU, double* SUn, double* SAUn,
                             cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ce_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ce_eig_smem());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int dmax_now = kh + ws.m;
  k_ce_formC<<<dmax_now, 256, 0, st>>>(ws, SU, kh);
  k_ce_rinv<<<dmax_now, 32, 0, st>>>(ws, kh);
  k_ce_M<<<dmax_now, 256, 0, st>>>(ws, kh);
  k_ce_svd<<<1, 512, 0, st>>>(ws, kh);
  k_ce_eig<<<1, 512, ce_eig_smem(), st>>>(ws);
  k_ce_invit<<<K_MAX, 256, 0, st>>>(ws);
  k_ce_finish<<<1, 512, 0, st>>>(ws, kh);
  k_ce_sketch_update<<<K_MAX, 512, 0, st>>>(ws, kh, SU, SAU, SUn, SAUn);
  return cudaGetLastError();
}

}  // namespace sdr
