// y = S x without any device allocation (sdr_sketch_noalloc in include/sdr.h).
//
// Some callers cannot let a library allocate device memory: code that runs
// while another component owns the device's memory (a framework's own pool or
// a fixed budget handed out at start-up), and latency-critical paths where a
// cudaMalloc, which may synchronise the device, is not acceptable.  For them
// this file applies the hash-defined sparse-sign embedding with all scratch in
// one file-scope device array (SCRATCH_WORDS 64-bit words, 8,256 bytes), which
// every GPU that loads the library holds until the process exits.  The caller
// supplies x and y; nothing else is needed (no handle, no index tables: each
// column's rows and signs are hashed on the fly).
//
// The arithmetic is the same exact fixed-point accumulation as the handle's
// sketch: per tile of columns the values are rounded to 2^-51 of the tile's
// largest magnitude, summed exactly per sketch row in 64-bit integers, and
// added into 128-bit accumulators inside a window fixed by max |x|.
#include <mutex>

#include "../../include/sdr.h"
#include "sdr_common.cuh"

namespace sdr {
namespace {

constexpr int NA_TILE = 1024;     // columns per tile (at most 2^12 keeps tile sums below 2^63)
constexpr int NA_THREADS = 256;
constexpr int NA_S_MAX = 512;    // sketch rows this entry point serves (its fixed scratch)
constexpr int NA_RPT = NA_S_MAX / NA_THREADS;
constexpr int SCRATCH_WORDS = 2 * NA_S_MAX + 64;  // 128-bit accumulators, then max|x|
constexpr int SC_MAX = 2 * NA_S_MAX;              // word holding the bits of max |x|
constexpr int64_t NA_MAX_N = 2147483647;       // columns are 31-bit indices

// The only device memory this entry point uses.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[SCRATCH_WORDS];

__global__ void k_na_clear(unsigned long long* sc, int s) {
  for (int i = threadIdx.x; i < 2 * s; i += blockDim.x) sc[i] = 0ull;
  if (threadIdx.x == 0) sc[SC_MAX] = 0ull;
}

__global__ void k_na_max(const double* __restrict__ x, int64_t n, unsigned long long* sc) {
  __shared__ unsigned long long red[32];
  unsigned long long m = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = abs_bits(x[i]);
    m = b > m ? b : m;
  }
  m = block_max_u64(m, red);
  if (threadIdx.x == 0 && m) atomicMax(sc + SC_MAX, m);
}

__global__ void __launch_bounds__(NA_THREADS) k_na_sketch(const double* __restrict__ x, int64_t n, int s,
                                                          int zeta, uint64_t seed, int win_bits,
                                                          unsigned long long* sc) {
  __shared__ double vals[NA_TILE];
  __shared__ unsigned long long acc_s[NA_S_MAX];
  __shared__ unsigned long long red[32];
  const double mx = __longlong_as_double((long long)sc[SC_MAX]);
  // x == 0: the cleared accumulators already hold S x.  A NaN or an Inf in x
  // (max |x| with exponent field 0x7FF) has no fixed-point window: nothing is
  // accumulated and k_na_finish writes NaN to every y[i].
  if (!(mx > 0.0) || bexp_of_bits(sc[SC_MAX]) == 0x7FF) return;
  const int top = window_top(mx, win_bits);
  unsigned long long lo[NA_RPT], hi[NA_RPT];
#pragma unroll
  for (int k = 0; k < NA_RPT; ++k) lo[k] = hi[k] = 0ull;
  for (int i = threadIdx.x; i < NA_S_MAX; i += blockDim.x) acc_s[i] = 0ull;
  const int64_t ntiles = (n + NA_TILE - 1) / NA_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t c0 = tile * NA_TILE;
    const int ncols = (int)(n - c0 < NA_TILE ? n - c0 : NA_TILE);
    unsigned long long mb = 0ull;
    for (int i = threadIdx.x; i < NA_TILE; i += blockDim.x) {
      const double v = i < ncols ? x[c0 + i] : 0.0;
      vals[i] = v;
      const unsigned long long b = abs_bits(v);
      mb = b > mb ? b : mb;
    }
    mb = block_max_u64(mb, red);  // synchronises the block
    const int emax = bexp_of_bits(mb);
    if (emax == 0 || emax == 0x7FF) continue;  // an all-zero tile adds nothing (uniform branch)
    for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
      const long long q = quantize_fixed(vals[i], emax);
      if (q == 0) continue;
      int rows[ZETA_MAX], sg[ZETA_MAX];
      sketch_column(seed, s, zeta, (uint64_t)(c0 + i), rows, sg);
      for (int k = 0; k < zeta; ++k)
        atomicAdd(&acc_s[rows[k]], (unsigned long long)(sg[k] < 0 ? -q : q));  // two's complement sum
    }
    __syncthreads();
    const int sh = (emax - 1022) - 51 - (top - 126);
#pragma unroll
    for (int k = 0; k < NA_RPT; ++k) {
      const int row = threadIdx.x + k * blockDim.x;
      if (row < s) {
        add_shifted128(lo[k], hi[k], (long long)acc_s[row], sh);
        acc_s[row] = 0ull;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < NA_RPT; ++k) {
    const int row = threadIdx.x + k * blockDim.x;
    if (row < s) atomic_add128(sc + 2 * row, lo[k], hi[k]);
  }
}

__global__ void k_na_finish(const unsigned long long* sc, int s, int win_bits, double scale, double* __restrict__ y) {
  const double mx = __longlong_as_double((long long)sc[SC_MAX]);
  if (bexp_of_bits(sc[SC_MAX]) == 0x7FF) {  // x holds a NaN or an Inf: S x is not finite
    for (int i = threadIdx.x; i < s; i += blockDim.x) y[i] = __longlong_as_double(0x7FF8000000000000ll);
    return;
  }
  const int top = window_top(mx > 0.0 ? mx : 1.0, win_bits);
  for (int i = threadIdx.x; i < s; i += blockDim.x)
    y[i] = mx > 0.0 ? int128_to_double(sc[2 * i], sc[2 * i + 1], top - 126) * scale : 0.0;
}

// Device address of the scratch array, looked up once per device (by the first
// call on that device, with it current) and kept for the life of the process.
// The cache is not refreshed after cudaDeviceReset: a caller that resets a
// device must not call this entry point again on it.
std::mutex g_mu;
unsigned long long* g_addr[128] = {};

cudaError_t scratch_address(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = (unsigned long long*)p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace sdr

extern "C" sdr_status sdr_sketch_noalloc(const double* x, int64_t n, int32_t s, int32_t zeta, uint64_t seed,
                                         double* y, void* stream) {
  using namespace sdr;
  if (!x || !y || n < 1 || n > NA_MAX_N || s < 1 || s > NA_S_MAX || zeta < 1 || zeta > s || zeta > ZETA_MAX)
    return SDR_ERR_INVALID_ARG;
  unsigned long long* sc = nullptr;
  if (scratch_address(&sc) != cudaSuccess) return SDR_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  int win_bits = 0;
  while (((int64_t)1 << win_bits) < n) ++win_bits;
  win_bits += 1;
  int nsm = 152;  // GB300, kept if the query below fails
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (n + NA_TILE - 1) / NA_TILE;
  const int g_sketch = (int)(ntiles < 4 * nsm ? ntiles : 4 * nsm);
  int64_t gm = (n + 255) / 256;
  if (gm > 4 * nsm) gm = 4 * nsm;
  k_na_clear<<<1, 512, 0, st>>>(sc, s);
  k_na_max<<<(int)gm, 256, 0, st>>>(x, n, sc);
  k_na_sketch<<<g_sketch, NA_THREADS, 0, st>>>(x, n, s, zeta, seed, win_bits, sc);
  k_na_finish<<<1, 512, 0, st>>>(sc, s, win_bits, 1.0 / std::sqrt((double)zeta), y);
  if (cudaGetLastError() != cudaSuccess) return SDR_ERR_CUDA;
  return SDR_OK;
}
