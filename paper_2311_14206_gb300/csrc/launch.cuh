// Host-side launchers of the GMRES-SDR kernels (one translation unit each).
#pragma once
#include "sdr_common.cuh"

namespace sdr {

struct CsrDev {
  int64_t n, nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const float* val32;  // FP32 copy of val (the refined form's inner solver), else null
};

// ---- sketch.cu ----
cudaError_t launch_sketch_build(const WS& ws, int64_t n, uint16_t* ent, uint16_t* ptr, cudaStream_t st);
// acc (+=) S_raw x for a vector whose entries are bounded by ctl->... ; the
// window top is read from *top_dev (device int) so producers can set it.
template <typename T>
cudaError_t launch_sketch_vec(const WS& ws, const T* x, int64_t n, unsigned long long* acc,
                              const int* top_dev, cudaStream_t st);
// y = scale * acc * 2^(top-126) / sqrt(zeta) for s rows; zeroes acc.
cudaError_t launch_sketch_finish(const WS& ws, unsigned long long* acc, const int* top_dev, double* y,
                                 cudaStream_t st);
// cos(pi m / (2n)) for m = 0 .. n into tab (the DCT sketch's cosine table).
cudaError_t launch_dct_table(double* tab, int64_t n, cudaStream_t st);
// *top_dev = window for max|x| (reduction over x).
template <typename T>
cudaError_t launch_maxabs_top(const WS& ws, const T* x, int64_t n, int* top_dev, cudaStream_t st);

// ---- arnoldi.cu ----
// Solve start: ||b||, max|b|, ||A||_inf, tol into ctl.
// Tall vectors hold T (double, or float for the refined form's inner solver).
template <typename T>
cudaError_t launch_solve_init_x(const WS& ws, CsrDev A, const T* b, const T* x, double rel_tol, cudaStream_t st,
                                bool keep_logs = false);
// r = b - A x into rout; ||r||, max|r| into ctl (res, rmax); S r into accR (window from
// ctl bmax + anorm_inf * xmax_bits).  mode 0: unconditional (solve start, x = x0);
// mode 1: only when ctl->check, and the last CTA applies the residual control.
template <typename T>
cudaError_t launch_residual(const WS& ws, CsrDev A, const T* b, const T* x, T* rout,
                            unsigned long long* accR, int j, int mode, cudaStream_t st);
// Arnoldi step j: w = A v_j with window dots; coefficients into ctl.
template <typename T>
cudaError_t launch_spmv_dots(const WS& ws, CsrDev A, const T* const* vcol, int j, cudaStream_t st);
// v_hat_{j+1} = a0 w - sum a_i v_i, with its norm, cross dots and max magnitude.
template <typename T>
cudaError_t launch_update_sketch(const WS& ws, const T* const* vcol, T* vnext, int j, cudaStream_t st);
// x_trial = x_cur + [U V(:,0:j+1)] (scaled ytil) when ctl->check.
template <typename T>
cudaError_t launch_check_gemv(const WS& ws, const T* U, const T* const* vcol, const T* xcur,
                              T* xtrial, int kh, int j, int ubuf, cudaStream_t st);
// U_new = [U V(:,0:jf)] P' (kprime columns from ctl).
template <typename T>
cudaError_t launch_recycle_gemm(const WS& ws, const T* U, const T* const* vcol, T* Unew,
                                int kh, int ucur, int unext, cudaStream_t st);
// U_new = [U V(:,0:jf)] P' on the tcgen05 tensor cores (float64 only; exact,
// bit-identical to the integer-pipe product).  v0 = V(:, 0), vs = V(:, 1..).
cudaError_t launch_recycle_tc(const WS& ws, const double* U, const double* v0, const double* vs, double* Unew,
                              int kh, int ucur, int unext, cudaStream_t st);
// y = A x (plain SpMV, used for A U in the exact recycling variant).
template <typename T>
cudaError_t launch_spmv(CsrDev A, const T* x, T* y, cudaStream_t st);
int update_grid(const WS& ws);
// Refined form: r32 = (float)r64 and d32 = 0; x64 += (double)d32.
cudaError_t launch_to_f32(const double* r64, float* r32, float* d32, int64_t n, cudaStream_t st);
cudaError_t launch_add_f32(double* x64, const float* d32, int64_t n, cudaStream_t st);
// S v_hat_j of the cycle's last column, with the column's finish.
template <typename T>
cudaError_t launch_sketch_col(const WS& ws, const T* x, int j, cudaStream_t st);

// ---- dense_step.cu ----
// Cycle start on the Arnoldi stream: Sr0, beta, SV(:,0), z = Sr0, control flags.
cudaError_t launch_cycle_head(const WS& ws, int kh, unsigned long long* accR, int persist_safety, cudaStream_t st);
// Cycle start on the control stream: QR of SAU (kh columns), z and sres.
cudaError_t launch_cycle_qr(const WS& ws, const double* SAU, int kh, cudaStream_t st);
// Arnoldi step j, small dense part: h(j+1,j), SV(:,j+1), SAV(:,j), QR update, sres, control.
cudaError_t launch_step_dense(const WS& ws, int j, int kh, int ubuf, unsigned long long* accR, cudaStream_t st);
// *flag = 1 when the sketched recycle block SAU (s x kd, kd <= K_MAX) is
// numerically rank-deficient (|R_pp| <= s eps max ||SAU(:, q)||), else 0.
cudaError_t launch_sau_rank(const double* SAU, int s, int kd, int* flag, cudaStream_t st);
// max |U(:, l)| of kdim columns into ctl->umax[ubuf] (after an import).
template <typename T>
cudaError_t launch_umax(const WS& ws, const T* U, int kdim, int ubuf, cudaStream_t st);

// ---- dense_cycle.cu ----
// Cycle end: harmonic-Ritz recycling (Section 3.5); P' into ws.P, SU/SAU for the next cycle.
// part 0..8: form C, R^{-1}, M (+ full-rank certificate), truncated SVD (only
// when not certified), FP32 eigenvalue candidates, FP64 inverse iteration per
// candidate, selection, basis + P, SU/SAU products.
constexpr int CYCLE_END_PARTS = 9;
cudaError_t launch_cycle_end_part(int part, const WS& ws, int kh, int ucur, const double* SU, const double* SAU,
                                  double* SUn, double* SAUn, cudaStream_t st);

}  // namespace sdr
