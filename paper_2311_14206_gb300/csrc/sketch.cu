// Sparse-sign embedding S (Section 3, eq. (sketch)): per-tile index tables and
// the exact fixed-point accumulation of S x.
//
// S is defined column by column by a counter-based hash (sketch_column in
// sdr_common.cuh).  For fast accumulation the columns are cut into tiles of
// TILE rows of x; for each tile the build kernel lists, per sketch row, the
// tile-local columns that hit that row (with their sign).  Applying S then is
// a gather per sketch row from the tile's values staged in shared memory:
// no atomics in shared memory and no FP64 additions.
//
// Accumulation: a tile's values are quantised to 2^-51 of the tile's largest
// magnitude (integer arithmetic on the bit pattern), summed exactly in int64
// per sketch row, shifted into a 128-bit window fixed by an a-priori bound on
// the vector, and added across CTAs with 64-bit integer atomics and an explicit
// carry.  Integer addition is associative, so S x is bit-for-bit reproducible.
#include "launch.cuh"

namespace sdr {

// One CTA per tile.  Shared: rows/signs of the tile (uint16 packed), counts,
// cursors.  Output order within a sketch row is by increasing column, so the
// table is deterministic.
__global__ void k_sketch_build(uint64_t seed, int s, int zeta, int64_t n, int tileR, uint16_t* ent,
                               uint16_t* ptr) {
  extern __shared__ unsigned char smem[];
  uint16_t* code = (uint16_t*)smem;                       // tileR*zeta: row | sign<<15
  int* cnt = (int*)(code + ((tileR * zeta + 1) & ~1));    // s+1
  int* cur = cnt + (S_MAX + 1);                           // s
  const int tile = blockIdx.x;
  const int64_t c0 = (int64_t)tile * tileR;
  const int ncols = (int)(n - c0 < (int64_t)tileR ? n - c0 : (int64_t)tileR);
  for (int i = threadIdx.x; i <= s; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
    int rows[ZETA_MAX], sg[ZETA_MAX];
    sketch_column(seed, s, zeta, (uint64_t)(c0 + i), rows, sg);
    for (int q = 0; q < zeta; ++q) {
      code[i * zeta + q] = (uint16_t)(rows[q] | (sg[q] < 0 ? 0x8000 : 0));
      atomicAdd(&cnt[rows[q]], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan (s <= 512)
    int acc = 0;
    for (int r = 0; r < s; ++r) {
      int c = cnt[r];
      cnt[r] = acc;
      cur[r] = acc;
      acc += c;
    }
    cnt[s] = acc;
  }
  __syncthreads();
  uint16_t* e = ent + (int64_t)tile * tileR * zeta;
  for (int i = threadIdx.x; i < ncols; i += blockDim.x) {
    for (int q = 0; q < zeta; ++q) {
      uint16_t cd = code[i * zeta + q];
      int row = cd & 0x7FFF;
      int pos = atomicAdd(&cur[row], 1);
      e[pos] = (uint16_t)(i | (cd & 0x8000));
    }
  }
  __syncthreads();
  // deterministic order: sort each row's list by column (insertion sort)
  for (int r = threadIdx.x; r < s; r += blockDim.x) {
    int a = cnt[r], b = cnt[r + 1];
    for (int x = a + 1; x < b; ++x) {
      uint16_t v = e[x];
      int y = x - 1;
      while (y >= a && (e[y] & 0x7FFF) > (v & 0x7FFF)) {
        e[y + 1] = e[y];
        --y;
      }
      e[y + 1] = v;
    }
  }
  uint16_t* p = ptr + (int64_t)tile * PTR_STRIDE;
  for (int r = threadIdx.x; r <= s; r += blockDim.x) p[r] = (uint16_t)cnt[r];
}

cudaError_t launch_sketch_build(const WS& ws, int64_t n, uint16_t* ent, uint16_t* ptr, cudaStream_t st) {
  int tileR = sketch_tile_rows(ws.zeta);
  int ntiles = (int)((n + tileR - 1) / tileR);
  size_t sm = (size_t)((tileR * ws.zeta + 1) & ~1) * 2 + (size_t)(2 * S_MAX + 1) * sizeof(int);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_sketch_build, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_sketch_build<<<ntiles, 512, sm, st>>>(ws.seed, ws.s, ws.zeta, n, tileR, ent, ptr);
  return cudaGetLastError();
}

// Generic S x with the window top read from device memory.
template <typename T>
__global__ void k_sketch_vec(WS ws, const T* __restrict__ x, int64_t n, unsigned long long* acc,
                             const int* top_dev) {
  extern __shared__ unsigned char smem[];
  const int tileR = sketch_tile_rows(ws.zeta);
  double* vals = (double*)smem;
  uint16_t* ent_s = (uint16_t*)(vals + tileR);
  uint16_t* ptr_s = ent_s + tileR * ws.zeta;
  __shared__ unsigned long long red[32];
  const int top = *top_dev;
  unsigned long long lo[SK_RPT], hi[SK_RPT];
#pragma unroll
  for (int k = 0; k < SK_RPT; ++k) lo[k] = hi[k] = 0ull;
  const int ntiles = (int)((n + tileR - 1) / tileR);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = (int64_t)tile * tileR;
    const int ncols = (int)(n - r0 < (int64_t)tileR ? n - r0 : (int64_t)tileR);
    if (!ws.sketch_kind) tile_sketch_prefetch(ws, tileR, tile, ent_s, ptr_s);
    for (int i = threadIdx.x; i < tileR; i += blockDim.x) vals[i] = i < ncols ? (double)x[r0 + i] : 0.0;
    if (ws.sketch_kind)
      tile_dct_accumulate<SK_RPT>(ws, r0, ncols, vals, top, lo, hi);
    else
      tile_sketch_accumulate<SK_RPT>(ws, ncols, vals, ent_s, ptr_s, red, top, lo, hi);
  }
#pragma unroll
  for (int k = 0; k < SK_RPT; ++k) {
    const int row = threadIdx.x + k * blockDim.x;
    if (row < ws.s) atomic_add128(acc + 2 * row, lo[k], hi[k]);
  }
}

template <typename T>
cudaError_t launch_sketch_vec(const WS& ws, const T* x, int64_t n, unsigned long long* acc,
                              const int* top_dev, cudaStream_t st) {
  size_t sm = sketch_smem_bytes(ws.zeta);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_sketch_vec<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sketch_smem_bytes(ZETA_MAX));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int tileR = sketch_tile_rows(ws.zeta);
  int ntiles = (int)((n + tileR - 1) / tileR);
  int grid = ntiles < ws.grid_max ? ntiles : ws.grid_max;
  if (grid < 1) grid = 1;
  k_sketch_vec<T><<<grid, SK_THREADS, sm, st>>>(ws, x, n, acc, top_dev);
  return cudaGetLastError();
}

__global__ void k_sketch_finish(WS ws, unsigned long long* acc, const int* top_dev, double* y) {
  const int top = *top_dev;
  for (int i = threadIdx.x; i < ws.s; i += blockDim.x) {
    y[i] = int128_to_double(acc[2 * i], acc[2 * i + 1], top - 126) * ws.inv_sqrt_zeta;
    acc[2 * i] = 0ull;
    acc[2 * i + 1] = 0ull;
  }
}

cudaError_t launch_sketch_finish(const WS& ws, unsigned long long* acc, const int* top_dev, double* y,
                                 cudaStream_t st) {
  k_sketch_finish<<<1, 512, 0, st>>>(ws, acc, top_dev, y);
  return cudaGetLastError();
}

// max|x| over a vector -> window top for a sketch of x (one CTA-level pass +
// last-CTA finish through an atomicMax on the bit pattern).
template <typename T>
__global__ void k_maxabs_top(WS ws, const T* __restrict__ x, int64_t n, unsigned long long* scratch,
                             int* top_dev) {
  __shared__ unsigned long long red[32];
  unsigned long long mb = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long b = abs_bits((double)x[i]);
    mb = b > mb ? b : mb;
  }
  mb = block_max_u64(mb, red);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    atomicMax(scratch, mb);
    __threadfence();
    unsigned int prev = atomicAdd((unsigned int*)(scratch + 1), 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    unsigned long long m = atomicAdd(scratch, 0ull);
    *top_dev = window_top(__longlong_as_double((long long)m), ws.win_bits);
    scratch[0] = 0ull;
    scratch[1] = 0ull;
  }
}

template <typename T>
cudaError_t launch_maxabs_top(const WS& ws, const T* x, int64_t n, int* top_dev, cudaStream_t st) {
  // scratch: two u64 words right after the 2*S_MAX words of the second accumulator block
  unsigned long long* scratch = ws.acc + 6 * S_MAX;
  int grid = (int)((n + 255) / 256);
  if (grid > ws.grid_max) grid = ws.grid_max;
  if (grid < 1) grid = 1;
  k_maxabs_top<T><<<grid, 256, 0, st>>>(ws, x, n, scratch, top_dev);
  return cudaGetLastError();
}

// Cosine table of the DCT sketch: tab[m] = cos(pi m / (2n)), m = 0 .. n.
__global__ void k_dct_table(double* tab, int64_t n) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m <= n; m += (int64_t)gridDim.x * blockDim.x)
    tab[m] = cospi((double)m / (double)(2 * n));
}

cudaError_t launch_dct_table(double* tab, int64_t n, cudaStream_t st) {
  int64_t g = (n + 256) / 256;
  if (g > 4096) g = 4096;
  k_dct_table<<<(int)g, 256, 0, st>>>(tab, n);
  return cudaGetLastError();
}

template cudaError_t launch_sketch_vec<double>(const WS&, const double*, int64_t, unsigned long long*, const int*,
                                               cudaStream_t);
template cudaError_t launch_sketch_vec<float>(const WS&, const float*, int64_t, unsigned long long*, const int*,
                                              cudaStream_t);
template cudaError_t launch_maxabs_top<double>(const WS&, const double*, int64_t, int*, cudaStream_t);
template cudaError_t launch_maxabs_top<float>(const WS&, const float*, int64_t, int*, cudaStream_t);

}  // namespace sdr
