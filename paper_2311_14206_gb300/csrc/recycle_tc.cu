// Recycle compression U_new = [U, V(:, 0:jf)] P'' (Algorithm 1, last block;
// Section 3.5) on the tcgen05 tensor cores, exact.
//
// The tall operand W = [U V] (N x d, d <= 160) and the small P'' (d x k', k'
// <= 32) are the same 52-bit fixed-point integers the integer-pipe kernel
// multiplies (column l of W scaled by 2^delta_l, unit 2^-51; P'' column q with
// exponent Pexp[q]).  Each integer X is split into seven signed base-256
// digits, X = sum_a x_a 256^a with x_a in [-128, 127] (the top digit in
// [-8, 8]), and likewise Y = sum_b y_b 256^b: this is the splitting of
// Ozaki, Ogita, Oishi and Rump (2012) with integer slices.  Every digit is
// exact in fp16, every digit product exact in fp32, and
//   X Y = sum_g 256^g  sum_{a+b=g} x_a y_b,   g = 0 .. 12.
// The MMA for digit a of W multiplies it by all seven digits of P'' at once
// (B = [y_0 .. y_6], N = 7 x 32) into TMEM columns starting at 32a, so the
// product with y_b lands in the columns of group a + b: the tensor core sums
// the pairs of a group.  A group's sum over d <= 160 columns stays below 2^24
// in magnitude (at most six pairs of full digits, 6 * 160 * 2^14 < 2^24), so
// the fp32 accumulation is exact.  The epilogue converts the 13 group sums to
// integers, forms the 128-bit sum sum_g 256^g acc_g (equal to the integer
// kernel's exact sum) and rounds it once: the result is bit-identical to the
// integer-pipe kernel's.
//
// One persistent CTA per SM (576 threads, warp-specialised):
//   warp 17 (lane 0)   loads 128-row x 16-column tiles of W into shared memory
//                      with 2D TMA copies (cp.async.bulk.tensor): one copy per
//                      chunk, from a tensor map over the V slab or over U;
//   warps 8-15         quantise and split them into the seven fp16 digit planes
//                      (K-major core matrices, no swizzle);
//   warp 16 (lane 0)   issues the tcgen05.mma (M = 128, N = 224, K = 16) and
//                      commits to mbarriers; the warp owns the TMEM allocation;
//   warps 0-7          read the 13 group accumulators from TMEM (row = lane;
//                      warps w and w + 4 share a lane quarter and split the
//                      output columns), combine, round and store U_new.
// Every wait on an mbarrier is bounded; a wait that runs out sets ctl->tc_error,
// the CTA stops issuing work, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "launch.cuh"
#include "eidot.cuh"

namespace sdr {
namespace {

constexpr int TC_M = 128;      // rows per tile (MMA M)
constexpr int TC_KC = 16;      // W columns per chunk (MMA K of fp16)
constexpr int TC_DIG = 7;      // base-256 digits of a 52-bit integer
constexpr int TC_NC = 32;      // output columns per digit block of B (K_MAX)
constexpr int TC_N = TC_DIG * TC_NC;        // 224: MMA N
constexpr int TC_GROUPS = 2 * TC_DIG - 1;   // 13 digit-pair groups
constexpr int TC_KPAD = D_MAX;              // 160: K extent of B
constexpr int TC_NSTG = 4;                  // staging buffers (fp64 tiles)
constexpr int TC_NAB = 3;                   // digit-plane buffers
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_THREADS = 576;             // 18 warps
constexpr int TC_EPI_WARPS = 8;             // warps 0-7
constexpr int TC_PRODUCERS = 256;           // warps 8-15
constexpr int TC_MMA_WARP = 16, TC_TMA_WARP = 17;

// shared-memory layout (bytes)
constexpr int B_ROWS_CM = TC_N / 8;                    // 28 core matrices per K block of B
constexpr int B_LBO = B_ROWS_CM * 128;                 // 3584: next K block of B
constexpr int B_BYTES = TC_N * TC_KPAD * 2;            // 71,680
constexpr int A_DIGIT_BYTES = TC_M * TC_KC * 2;        // 4,096 per digit plane
constexpr int A_LBO = (TC_M / 8) * 128;                // 2048: second K block of a plane
constexpr int A_BUF_BYTES = TC_DIG * A_DIGIT_BYTES;    // 28,672
constexpr int STG_COL_BYTES = TC_M * 8;                // 1,024: one column segment
constexpr int STG_BYTES = TC_KC * STG_COL_BYTES;       // 16,384
constexpr int OFF_B = 0;
constexpr int OFF_A = OFF_B + B_BYTES;
constexpr int OFF_Z = OFF_A + TC_NAB * A_BUF_BYTES;
constexpr int OFF_STG = OFF_Z + A_DIGIT_BYTES;
constexpr int TC_SMEM = OFF_STG + TC_NSTG * STG_BYTES + 128;  // + slack to align the base to 128 bytes
static_assert(TC_SMEM + 1536 <= 227 * 1024, "shared memory of the tensor-core recycle kernel");
constexpr long long TC_SPIN = 4000000000LL;  // clock cycles (about two seconds) per wait

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: K-major core matrices of 8 rows x
// 16 bytes, no swizzle; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups; bit 46 is the sm_100-family version field.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: fp32 accumulator (bit 4), fp16 A and B
// (format fields 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t TC_IDESC = (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(saddr(b)), "r"(parity)
               : "memory");
  return ok != 0;
}
// Bounded wait: false when the CTA aborted (here or in another role).
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!bar_test(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > TC_SPIN) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// 2D TMA copy of the box at (x = first row, y = first column) of a tensor map
// into shared memory; rows and columns outside the map are filled with zeros.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}

// The integer kernel's operand quantisation (q52 with emax 1022) as one
// signed 64-bit value v, |v| <= 2^51.
__device__ __forceinline__ long long q52_value(double x, int delta) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int sh = 1024 - (ex + delta);
  if (ex == 0 || sh >= 60) return 0;
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const long long q = (long long)((mant + (1ull << (sh - 1))) >> sh);
  return (b >> 63) ? -q : q;
}

// Adding 128 at every digit position makes the digits of v non-negative:
// byte a of u = v + OFFSET is x_a + 128 for the balanced digits x_a.
constexpr unsigned long long DIGIT_OFFSET = 0x0080808080808080ull;

// Two fp16 digits in one word: byte a of the words w0 and w1 (the 32-bit half
// of u that holds byte a) as the halves 0x6400 | byte = 1024 + byte, minus
// 1024 + 128 in one packed subtraction (exact: integers below 2048).
__device__ __forceinline__ uint32_t digit_pair_f16(uint32_t w0, uint32_t w1, int a3) {
  const uint32_t p = __byte_perm(w0, w1, (uint32_t)a3 | ((uint32_t)(4 + a3) << 8));
  const uint32_t h = (p & 0x00FF00FFu) | 0x64006400u;
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(h), "r"(0x64806480u));
  return r;
}

__device__ __forceinline__ int column_delta(const Ctl* c, int ubuf, int kh, int l) {
  const unsigned long long mb = l < kh ? c->umax[ubuf][l] : c->vmax[l - kh];
  const int e = bexp_of_bits(mb);
  return e == 0 ? 0 : -(e - 1022);
}

// The K order of the MMA: nV chunks of 16 columns of the V slab (V(:, 0) is
// copied into the slab's front column before the launch, so V(:, 0:jf) is
// contiguous), then nU chunks of U.  Slot l' of that order holds column
// wcol(l') of W = [U, V(:, 0:jf)], or nothing (-1) in the padding.
__device__ __forceinline__ int slot_column(int lp, int nV, int kh, int jf) {
  if (lp < nV * TC_KC) return lp < jf ? kh + lp : -1;
  const int j = lp - nV * TC_KC;
  return j < kh ? j : -1;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_recycle_tc(WS ws, const __grid_constant__ CUtensorMap mapV, const __grid_constant__ CUtensorMap mapU,
                 double* __restrict__ Unew, int kh, int ucur, int unext) {
  Ctl* c = ws.ctl;
  const int kp = c->kprime, jf = c->jf;
  if (kp <= 0 || jf <= 0) return;
  const int d = kh + jf;
  const int nV = (jf + TC_KC - 1) / TC_KC, nU = (kh + TC_KC - 1) / TC_KC;
  if ((nV + nU) * TC_KC > TC_KPAD || kp > TC_NC) {  // cannot happen (jf <= M_MAX, kh <= K_MAX, kp <= K_MAX)
    if (threadIdx.x == 0 && blockIdx.x == 0) c->tc_error = 1;
    return;
  }
  extern __shared__ __align__(128) unsigned char tc_raw[];
  unsigned char* tc_smem = tc_raw + ((128u - (saddr(tc_raw) & 127u)) & 127u);  // 128-byte aligned (TMA)
  __shared__ __align__(8) uint64_t stg_full[TC_NSTG], stg_empty[TC_NSTG], a_full[TC_NAB], a_empty[TC_NAB];
  __shared__ __align__(8) uint64_t acc_full, acc_empty;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ int dl[TC_KPAD];    // per K slot: 2^delta scale of its W column
  __shared__ int slot_ok[TC_KPAD];
  __shared__ int fx[TC_NC];
  __shared__ unsigned int um_s[TC_NC];  // high words of max |U_new(:, q)| (only the exponent is used)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ld = ws.ldv, n = ws.n;
  const int64_t ntiles = (n + TC_M - 1) / TC_M;
  const int nkc = nV + nU;
  (void)d;

  // ---- set-up: scales, B = the seven digit planes of P'', the zero tile, barriers
  for (int lp = tid; lp < TC_KPAD; lp += blockDim.x) {
    const int l = slot_column(lp, nV, kh, jf);
    dl[lp] = l >= 0 ? column_delta(c, ucur, kh, l) : 0;
    slot_ok[lp] = l >= 0 ? 1 : 0;
  }
  for (int q = tid; q < TC_NC; q += blockDim.x) {
    fx[q] = q < kp ? ws.Pexp[q] : 0;
    um_s[q] = 0u;
  }
  {
    uint16_t* B = (uint16_t*)(tc_smem + OFF_B);  // fp16 bit patterns
    for (int idx = tid; idx < TC_KPAD * TC_NC; idx += blockDim.x) {
      const int lp = idx / TC_NC, q = idx % TC_NC;
      const int l = slot_column(lp, nV, kh, jf);
      long long v = 0;
      if (l >= 0 && q < kp) {
        const unsigned long long b = ws.Pq[l + (int64_t)q * D_MAX];  // packed (hi << 32) | lo, value hi 2^26 + lo
        v = (long long)(int)(b >> 32) * 67108864ll + (long long)(b & 0xFFFFFFFFull);
      }
      const unsigned long long u = (unsigned long long)v + DIGIT_OFFSET;
#pragma unroll
      for (int a = 0; a < TC_DIG; ++a) {
        const int row = TC_NC * a + q;  // B row: digit a of output column q
        const int off = ((lp >> 3) * B_ROWS_CM + (row >> 3)) * 64 + (row & 7) * 8 + (lp & 7);
        const int digit = (int)((u >> (8 * a)) & 0xFF) - 128;
        B[off] = __half_as_ushort(__int2half_rn(digit));
      }
    }
  }
  for (int i = tid; i < A_DIGIT_BYTES / 16; i += blockDim.x) ((uint4*)(tc_smem + OFF_Z))[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int i = 0; i < TC_NSTG; ++i) {
      bar_init(&stg_full[i], 1);
      bar_init(&stg_empty[i], TC_PRODUCERS / 32);
    }
    for (int i = 0; i < TC_NAB; ++i) {
      bar_init(&a_full[i], TC_PRODUCERS / 32);
      bar_init(&a_empty[i], 1);
    }
    bar_init(&acc_full, 1);
    bar_init(&acc_empty, TC_EPI_WARPS);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B and the zero tile: generic writes, async reads
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == TC_TMA_WARP) {
    // ---- bulk copies of W tiles into the staging ring
    if (lane == 0) {
      uint32_t sc = 0;
      const uint32_t stg0 = saddr(tc_smem + OFF_STG);
      for (int64_t tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
        const int r0 = (int)(tile * TC_M);
        for (int kc = 0; kc < nkc; ++kc, ++sc) {
          const int slot = (int)(sc % TC_NSTG);
          if (!bar_wait(&stg_empty[slot], ((sc / TC_NSTG) & 1) ^ 1, &abort_flag)) break;
          bar_arrive_tx(&stg_full[slot], STG_BYTES);  // the whole box, out-of-range parts zero-filled
          const uint32_t dst = stg0 + (uint32_t)(slot * STG_BYTES);
          if (kc < nV)
            tma_load_2d(dst, &mapV, r0, kc * TC_KC, &stg_full[slot]);
          else
            tma_load_2d(dst, &mapU, r0, (kc - nV) * TC_KC, &stg_full[slot]);
        }
      }
    }
  } else if (warp >= 8 && warp < 16) {
    // ---- quantise and split into digit planes
    const int pt = tid - 256, r = pt % TC_M, cg = pt / TC_M;  // row, column group (8 columns)
    uint32_t sc = 0, ac = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
      const int64_t r0 = tile * TC_M;
      const int nr = (int)(n - r0 < TC_M ? n - r0 : TC_M);
      bool ok = true;
      for (int kc = 0; kc < nkc && ok; ++kc, ++sc, ++ac) {
        const int slot = (int)(sc % TC_NSTG);
        if (!bar_wait(&stg_full[slot], (sc / TC_NSTG) & 1, &abort_flag)) { ok = false; break; }
        const double* stg = (const double*)(tc_smem + OFF_STG + slot * STG_BYTES);
        uint32_t ulo[8], uhi[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int cl = 8 * cg + i, lp = kc * TC_KC + cl;
          long long v = 0;
          if (slot_ok[lp] && r < nr) v = q52_value(stg[cl * TC_M + r], dl[lp]);
          const unsigned long long u = (unsigned long long)v + DIGIT_OFFSET;
          ulo[i] = (uint32_t)u;
          uhi[i] = (uint32_t)(u >> 32);
        }
        __syncwarp();
        if (lane == 0) bar_arrive(&stg_empty[slot]);
        const int ab = (int)(ac % TC_NAB);
        if (!bar_wait(&a_empty[ab], ((ac / TC_NAB) & 1) ^ 1, &abort_flag)) { ok = false; break; }
        unsigned char* A = tc_smem + OFF_A + ab * A_BUF_BYTES + (cg * (TC_M / 8) + (r >> 3)) * 128 + (r & 7) * 16;
#pragma unroll
        for (int a = 0; a < TC_DIG; ++a) {
          const uint32_t* w = a < 4 ? ulo : uhi;
          uint4 pk;
          pk.x = digit_pair_f16(w[0], w[1], a & 3);
          pk.y = digit_pair_f16(w[2], w[3], a & 3);
          pk.z = digit_pair_f16(w[4], w[5], a & 3);
          pk.w = digit_pair_f16(w[6], w[7], a & 3);
          *(uint4*)(A + a * A_DIGIT_BYTES) = pk;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) bar_arrive(&a_full[ab]);
      }
    }
  } else if (warp == TC_MMA_WARP) {
    // ---- MMA issue
    if (lane == 0) {
      uint32_t ac = 0, tt = 0;
      const uint32_t b0 = saddr(tc_smem + OFF_B), a0 = saddr(tc_smem + OFF_A), z0 = saddr(tc_smem + OFF_Z);
      for (int64_t tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x, ++tt) {
        if (!bar_wait(&acc_empty, (tt & 1) ^ 1, &abort_flag)) break;
        tc_fence_after();
        // zero the group columns the digit-0 MMA does not initialise
        mma_f16(tmem + TC_N, smem_desc(z0, A_LBO, 128), smem_desc(b0, B_LBO, 128), 0u);
        bool ok = true;
        for (int kc = 0; kc < nkc; ++kc, ++ac) {
          const int ab = (int)(ac % TC_NAB);
          if (!bar_wait(&a_full[ab], (ac / TC_NAB) & 1, &abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint64_t bdesc = smem_desc(b0 + (uint32_t)(2 * kc * B_LBO), B_LBO, 128);
#pragma unroll
          for (int a = 0; a < TC_DIG; ++a) {
            const uint64_t adesc = smem_desc(a0 + (uint32_t)(ab * A_BUF_BYTES + a * A_DIGIT_BYTES), A_LBO, 128);
            mma_f16(tmem + (uint32_t)(TC_NC * a), adesc, bdesc, (kc > 0 || a > 0) ? 1u : 0u);
          }
          mma_commit(&a_empty[ab]);
        }
        if (!ok) break;
        mma_commit(&acc_full);
      }
    }
    __syncwarp();
  } else if (warp < TC_EPI_WARPS) {
    // ---- epilogue: TMEM lanes 32 (w % 4) .. + 31 = rows of the tile; warps w
    // and w + 4 take alternate blocks of 8 output columns
    uint32_t tt = 0;
    const int quad = warp & 3, half = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16);
    for (int64_t tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x, ++tt) {
      if (!bar_wait(&acc_full, tt & 1, &abort_flag)) break;
      tc_fence_after();
      const int64_t r0 = tile * TC_M;
      const int nr = (int)(n - r0 < TC_M ? n - r0 : TC_M);
      const int r = 32 * quad + lane;
      for (int q0 = 8 * half; q0 < kp; q0 += 16) {
#pragma unroll
        for (int h4 = 0; h4 < 8; h4 += 4) {
          if (q0 + h4 >= kp) break;  // warp-uniform
          uint32_t g[TC_GROUPS][4];
#pragma unroll
          for (int gi = 0; gi < TC_GROUPS; ++gi) tmem_ld4(lane_base + (uint32_t)(TC_NC * gi + q0 + h4), g[gi]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int q = q0 + h4 + i;
            uint32_t um = 0u;
            if (q < kp && r < nr) {
              int a[TC_GROUPS];
#pragma unroll
              for (int gi = 0; gi < TC_GROUPS; ++gi) a[gi] = __float2int_rn(__uint_as_float(g[gi][i]));
              // four partial sums of four groups each (|.| < 2^49), then 128 bits
              const long long c0 = (long long)a[0] + (long long)a[1] * 256ll + (long long)a[2] * 65536ll +
                                   (long long)a[3] * 16777216ll;
              const long long c1 = (long long)a[4] + (long long)a[5] * 256ll + (long long)a[6] * 65536ll +
                                   (long long)a[7] * 16777216ll;
              const long long c2 = (long long)a[8] + (long long)a[9] * 256ll + (long long)a[10] * 65536ll +
                                   (long long)a[11] * 16777216ll;
              const long long c3 = (long long)a[12];
              unsigned long long lo = (unsigned long long)c0, hi = (unsigned long long)(c0 >> 63);
              const unsigned long long t = (unsigned long long)c1 << 32;
              lo += t;
              hi += (unsigned long long)(c1 >> 32) + (lo < t ? 1ull : 0ull);
              hi += (unsigned long long)c2 + ((unsigned long long)c3 << 32);
              const double v = i128_to_double(lo, hi, -102 + fx[q]);
              Unew[r0 + r + (int64_t)q * ld] = v;
              um = (uint32_t)(abs_bits(v) >> 32);
            }
            // column maximum of |U_new| (the next cycle's scale of this column)
            um = __reduce_max_sync(0xffffffffu, um);
            if (lane == 0 && um) atomicMax(&um_s[q], um);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(&acc_empty);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TC_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
  if (tid < kp && um_s[tid]) atomicMax(&c->umax[unext][tid], (unsigned long long)um_s[tid] << 32);
  if (tid == 0 && abort_flag) c->tc_error = 1;
}

}  // namespace

namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// 2D tensor map over n rows x cols columns (leading dimension ld) of float64,
// boxes of 128 rows x 16 columns, no swizzle, zero fill outside.
cudaError_t make_map(CUtensorMap* map, const double* base, int64_t n, int64_t cols, int64_t ld) {
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(double)};
  const cuuint32_t box[2] = {(cuuint32_t)TC_M, (cuuint32_t)TC_KC};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)base, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_recycle_tc(const WS& ws, const double* U, const double* v0, const double* vs, double* Unew,
                              int kh, int ucur, int unext, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_recycle_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // V(:, 0) into the slab's front column, so that the V part of W is one 2D array
  double* front = (double*)vs - ws.ldv;
  cudaError_t e = cudaMemcpyAsync(front, v0, (size_t)ws.n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  CUtensorMap mapV, mapU;
  e = make_map(&mapV, front, ws.n, (int64_t)ws.m + 1, ws.ldv);
  if (e != cudaSuccess) return e;
  e = make_map(&mapU, U, ws.n, ws.kmax, ws.ldv);
  if (e != cudaSuccess) return e;
  const int nsm = ws.grid_max / 8;
  const int64_t ntiles = (ws.n + TC_M - 1) / TC_M;
  const int grid = (int)(ntiles < nsm ? ntiles : nsm);
  k_recycle_tc<<<grid > 0 ? grid : 1, TC_THREADS, TC_SMEM, st>>>(ws, mapV, mapU, Unew, kh, ucur, unext);
  return cudaGetLastError();
}

}  // namespace sdr
