// Pieces of the differentiable solve (the adjoint form): the transposed
// sparsity pattern, the values of A^T in it, and the gradient of a loss with
// respect to the stored values of A.
//
// For x = A^{-1} b and a loss L(x), the adjoint method solves
// A^T lambda = dL/dx; then dL/db = lambda and dL/dA_ij = -lambda_i x_j on the
// stored entries.  The transposed system is solved by a second GMRES-SDR
// handle, which keeps its own recycle space from one call to the next.
#include "../../include/sdr.h"
#include "launch.cuh"

namespace sdr {
namespace {

__global__ void k_count_cols(const int32_t* __restrict__ col, int64_t nnz, int32_t* __restrict__ cnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[p]], 1);
}

// rowptrT = exclusive scan of cnt (n entries) with rowptrT[n] = nnz; one CTA,
// chunk by chunk; cursor = a copy of rowptrT(0:n).
__global__ void k_scan(const int32_t* __restrict__ cnt, int64_t n, int32_t* __restrict__ rowptrT,
                       int32_t* __restrict__ cursor) {
  __shared__ int32_t part[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int32_t v = i < n ? cnt[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // Hillis-Steele inclusive scan
      const int32_t add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) {
      const int32_t ex = carry + part[threadIdx.x] - v;
      rowptrT[i] = ex;
      cursor[i] = ex;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) rowptrT[n] = carry;
}

__global__ void k_scatter(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                          int32_t* __restrict__ cursor, int32_t* __restrict__ colT, int32_t* __restrict__ perm) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      const int32_t q = atomicAdd(&cursor[col[p]], 1);
      colT[q] = (int32_t)r;
      perm[q] = p;
    }
  }
}

// Each transposed row sorted by column (insertion sort), so the pattern does
// not depend on the order of the scatter's atomics.
__global__ void k_sort_rows(const int32_t* __restrict__ rowptrT, int64_t n, int32_t* __restrict__ colT,
                            int32_t* __restrict__ perm) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = rowptrT[r], b = rowptrT[r + 1];
    for (int32_t i = a + 1; i < b; ++i) {
      const int32_t c = colT[i], pv = perm[i];
      int32_t y = i - 1;
      while (y >= a && colT[y] > c) {
        colT[y + 1] = colT[y];
        perm[y + 1] = perm[y];
        --y;
      }
      colT[y + 1] = c;
      perm[y + 1] = pv;
    }
  }
}

__global__ void k_gather(const double* __restrict__ val, const int32_t* __restrict__ perm, int64_t nnz,
                         double* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = val[perm[q]];
}

// grad(p) = -lambda(i) x(col(p)) for the entries p of row i.
__global__ void k_value_grad(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t n,
                             const double* __restrict__ lam, const double* __restrict__ x,
                             double* __restrict__ grad) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double li = -lam[r];
    for (int32_t p = rowptr[r]; p < rowptr[r + 1]; ++p) grad[p] = li * x[col[p]];
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  return g < 1 ? 1 : (int)g;
}

}  // namespace
}  // namespace sdr

using namespace sdr;

extern "C" {

sdr_status sdr_csr_transpose(const sdr_csr* A, int32_t* rowptrT, int32_t* colT, int32_t* perm, int32_t* work,
                             void* stream) {
  if (!A || A->n <= 0 || A->nnz < 0 || A->nnz >= ((int64_t)1 << 31) || A->n >= ((int64_t)1 << 31) || !A->rowptr ||
      !A->col || !rowptrT || !colT || !perm || !work)
    return SDR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = A->n, nnz = A->nnz;
  int32_t* cnt = work;         // n
  int32_t* cursor = work + n;  // n
  if (cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int32_t), st) != cudaSuccess) return SDR_ERR_CUDA;
  if (nnz > 0) k_count_cols<<<grid_for(nnz), 256, 0, st>>>(A->col, nnz, cnt);
  k_scan<<<1, 1024, 0, st>>>(cnt, n, rowptrT, cursor);
  k_scatter<<<grid_for(n), 256, 0, st>>>(A->rowptr, A->col, n, cursor, colT, perm);
  k_sort_rows<<<grid_for(n), 256, 0, st>>>(rowptrT, n, colT, perm);
  return cudaGetLastError() == cudaSuccess ? SDR_OK : SDR_ERR_CUDA;
}

sdr_status sdr_gather_values(const double* val, const int32_t* perm, int64_t nnz, double* out, void* stream) {
  if (!val || !perm || !out || nnz < 0) return SDR_ERR_INVALID_ARG;
  if (nnz == 0) return SDR_OK;
  k_gather<<<grid_for(nnz), 256, 0, (cudaStream_t)stream>>>(val, perm, nnz, out);
  return cudaGetLastError() == cudaSuccess ? SDR_OK : SDR_ERR_CUDA;
}

sdr_status sdr_value_gradient(const sdr_csr* A, const double* lambda, const double* x, double* grad,
                              void* stream) {
  if (!A || A->n <= 0 || !A->rowptr || !A->col || !lambda || !x || !grad) return SDR_ERR_INVALID_ARG;
  k_value_grad<<<grid_for(A->n), 256, 0, (cudaStream_t)stream>>>(A->rowptr, A->col, A->n, lambda, x, grad);
  return cudaGetLastError() == cudaSuccess ? SDR_OK : SDR_ERR_CUDA;
}

}  // extern "C"
