// C ABI of the GMRES-SDR solver (include/sdr.h): handle, workspace and the
// host-side driver that issues one restart cycle after another.
//
// Control decisions inside a cycle (when to evaluate the true residual, when
// the cycle stops) are taken on the device from the control block; the host
// launches the m steps of a cycle back to back and synchronises once per
// cycle to read the outcome (converged, recycle dimension).
#include <cstdio>
#include <cstring>
#include <cmath>
#include <cstddef>
#include <memory>
#include <vector>

#include "../../include/sdr.h"
#include "launch.cuh"

namespace sdr {
size_t ce_scratch_doubles();
}

using namespace sdr;

// Per-launch CUDA-event timing (enabled by sdr_profile).
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<int> cls;   // class of event pair i (events 2i, 2i+1)
  std::vector<int> strm;  // stream of event pair i: 0 main, 1 control, 2 other
  double total_ms[SDR_K_COUNT] = {};
  int launches[SDR_K_COUNT] = {};
  // trace: every launch's start and end against one reference event
  int trace_cap = 0;
  cudaEvent_t ref = nullptr;
  bool ref_set = false;
  std::vector<sdr_trace_entry> trace;
};

struct sdr_handle {
  sdr_params p;
  int64_t n_max;
  cudaStream_t ust;  // the caller's stream: every call is ordered after earlier work on it
  cudaStream_t st = nullptr;   // the handle's main stream: Arnoldi kernels and everything outside a cycle
  cudaEvent_t evIn = nullptr, evOut = nullptr;  // fork from / join into the caller's stream
  cudaStream_t st2 = nullptr;  // control stream: dense steps and true-residual checks
  std::vector<cudaEvent_t> evS;  // evS[j]: step j's SpMV (column j sketched and finished)
  std::vector<cudaEvent_t> evD;  // evD[j]: dense step j and its check
  cudaEvent_t evFork = nullptr, evJoin = nullptr;
  int device;
  WS ws;
  std::vector<void*> allocs;
  uint16_t* sk_ent = nullptr;
  uint16_t* sk_ptr = nullptr;
  int cu = 0;  // current recycle buffer
  int kh = 0;  // current recycle dimension
  std::vector<double> hist;
  std::vector<double> hist_givens;  // (sine, cosine) per step
  std::vector<CycleLog> log;
  double* d_tmp = nullptr;  // n_max scratch vector (A u)
  Prof prof;
  int launches = 0;  // kernels launched by the current call
  int sau_refreshes = 0;   // stale_check: SAU recomputations in the current sdr_solve
  int extra_matvecs = 0;   // products with A outside the cycles' own count (those recomputations)
  int prec = SDR_PREC_F64;   // storage type of the tall arrays: double, or float (refined form)
  void* rhs32 = nullptr;     // refined form: float32 right-hand side of the inner solve
  void* dx32 = nullptr;      // refined form: float32 inner solution
  Ctl* hc = nullptr;         // pinned host copy of the control block, read after each cycle
  // Cycle graphs.  A cycle's launch sequence depends only on (kh, cu, rb) and
  // on the buffers it touches; the caller's A, b and x are first copied into
  // handle-owned staging buffers so that one captured graph per state serves
  // every later solve of the same size.
  bool use_graphs = true;
  int32_t* st_rowptr = nullptr;
  int32_t* st_col = nullptr;
  double* st_val = nullptr;
  float* st_val32 = nullptr;
  int64_t st_nnz_cap = 0;
  double* st_b = nullptr;
  double* st_x = nullptr;
  struct GraphEntry {
    int64_t n, nnz;
    int kh, cu, rb, xpar, kernels;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
};

namespace {

sdr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SDR_OK;
  if (e == cudaErrorMemoryAllocation) return SDR_ERR_OOM;
  return SDR_ERR_CUDA;
}

#define SDR_CK(x)                                   \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return cuda_status(e_);  \
  } while (0)

template <typename T>
cudaError_t halloc(sdr_handle* h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *p = (T*)q;
  return cudaSuccess;
}

int ceil_log2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}

bool csr_ok(const sdr_handle* h, const sdr_csr* A) {
  return A && A->n > 0 && A->n <= h->n_max && A->nnz >= 0 && A->rowptr && A->col && A->val &&
         A->nnz < ((int64_t)1 << 31) && (h->prec == SDR_PREC_F64 || A->val32) &&
         (h->ws.sketch_kind == 0 || A->n == h->ws.dct_n);  // a DCT sketch is drawn for one size
}

CsrDev to_dev(const sdr_csr* A) { return CsrDev{A->n, A->nnz, A->rowptr, A->col, A->val, A->val32}; }

// Column c of a tall array of element type T with leading dimension ld.
template <typename T>
T* tall_col(void* base, int64_t ld, int64_t c) {
  return (T*)base + c * ld;
}

int* ctl_int_field(Ctl* c, size_t off) { return (int*)((char*)c + off); }

// Kernels issued by each launcher (for the launch count).
constexpr int kKernelsPerClass[SDR_K_COUNT] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 4, 1, 1, 1, 1, 1, 2, 1, 1, 1, 1};

cudaError_t prof_begin(sdr_handle* h, int cls, cudaStream_t st) {
  h->launches += kKernelsPerClass[cls];
  if (!h->prof.on) return cudaSuccess;
  Prof& P = h->prof;
  while (P.pool.size() < 2 * (P.cls.size() + 1)) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    P.pool.push_back(e);
  }
  P.cls.push_back(cls);
  P.strm.push_back(st == h->st ? 0 : (st == h->st2 ? 1 : 2));
  if (P.trace_cap > 0 && !P.ref_set) {
    cudaError_t r = cudaEventRecord(P.ref, st);
    if (r != cudaSuccess) return r;
    P.ref_set = true;
  }
  return cudaEventRecord(P.pool[2 * (P.cls.size() - 1)], st);
}

cudaError_t prof_end(sdr_handle* h, cudaStream_t st) {
  if (!h->prof.on) return cudaSuccess;
  return cudaEventRecord(h->prof.pool[2 * (h->prof.cls.size() - 1) + 1], st);
}

// Fold the recorded event pairs into the totals (stream must be idle).
cudaError_t prof_collect(sdr_handle* h) {
  Prof& P = h->prof;
  if (!P.on) return cudaSuccess;
  for (size_t i = 0; i < P.cls.size(); ++i) {
    float ms = 0.f;
    cudaError_t r = cudaEventElapsedTime(&ms, P.pool[2 * i], P.pool[2 * i + 1]);
    if (r != cudaSuccess) return r;
    P.total_ms[P.cls[i]] += ms;
    P.launches[P.cls[i]] += 1;
    if (P.trace_cap > 0 && (int)P.trace.size() < P.trace_cap) {
      float t0 = 0.f, t1 = 0.f;
      r = cudaEventElapsedTime(&t0, P.ref, P.pool[2 * i]);
      if (r == cudaSuccess) r = cudaEventElapsedTime(&t1, P.ref, P.pool[2 * i + 1]);
      if (r != cudaSuccess) return r;
      sdr_trace_entry te;
      te.cls = P.cls[i];
      te.stream = P.strm[i];
      te.start_us = 1e3 * (double)t0;
      te.end_us = 1e3 * (double)t1;
      P.trace.push_back(te);
    }
  }
  P.cls.clear();
  P.strm.clear();
  return cudaSuccess;
}

#define SDR_LAUNCH_ON(h, cls, stream, call)    \
  do {                                         \
    SDR_CK(prof_begin((h), (cls), (stream)));  \
    SDR_CK(call);                              \
    SDR_CK(prof_end((h), (stream)));           \
  } while (0)
#define SDR_LAUNCH(h, cls, call) SDR_LAUNCH_ON(h, cls, (h)->st, call)

// A call's work runs on the handle's own streams (a legacy default stream
// cannot be captured into a graph); it starts after the work already queued
// on the caller's stream and the caller's stream waits for it on return.
struct StreamGuard {
  sdr_handle* h;
  explicit StreamGuard(sdr_handle* hh) : h(hh) {
    if (cudaEventRecord(h->evIn, h->ust) == cudaSuccess) cudaStreamWaitEvent(h->st, h->evIn, 0);
  }
  ~StreamGuard() {
    if (cudaEventRecord(h->evOut, h->st) == cudaSuccess) cudaStreamWaitEvent(h->ust, h->evOut, 0);
  }
  StreamGuard(const StreamGuard&) = delete;
  StreamGuard& operator=(const StreamGuard&) = delete;
};

}  // namespace

template <typename T>
static sdr_status issue_sau(sdr_handle* h, const sdr_csr* A, int64_t n);
static sdr_status verify_sau_rank(sdr_handle* h);

extern "C" {

int32_t sdr_abi_version(void) { return SDR_ABI_VERSION; }

const char* sdr_status_string(sdr_status st) {
  switch (st) {
    case SDR_OK: return "ok";
    case SDR_ERR_INVALID_ARG: return "invalid argument";
    case SDR_ERR_CUDA: return "CUDA error";
    case SDR_ERR_OOM: return "out of device memory";
    case SDR_ERR_NOT_CONVERGED: return "not converged within max_cycles";
    case SDR_ERR_BREAKDOWN: return "Arnoldi breakdown without convergence";
    case SDR_ERR_RANK: return "sketched least-squares matrix lost rank";
    case SDR_ERR_NOT_IMPLEMENTED: return "not implemented";
  }
  return "unknown status";
}

sdr_status sdr_destroy(sdr_handle* h) {
  if (!h) return SDR_OK;
  if (h->st2) cudaStreamSynchronize(h->st2);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  if (h->prof.ref) cudaEventDestroy(h->prof.ref);
  for (cudaEvent_t e : h->evS) cudaEventDestroy(e);
  for (cudaEvent_t e : h->evD) cudaEventDestroy(e);
  if (h->evFork) cudaEventDestroy(h->evFork);
  if (h->evJoin) cudaEventDestroy(h->evJoin);
  if (h->st) cudaStreamSynchronize(h->st);
  if (h->st2) cudaStreamDestroy(h->st2);
  if (h->st) cudaStreamDestroy(h->st);
  if (h->evIn) cudaEventDestroy(h->evIn);
  if (h->evOut) cudaEventDestroy(h->evOut);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  if (h->hc) cudaFreeHost(h->hc);
  cudaFree(h->st_col);
  cudaFree(h->st_val);
  cudaFree(h->st_val32);
  for (void* q : h->allocs) cudaFree(q);
  delete h;
  return SDR_OK;
}

sdr_status sdr_create(const sdr_params* p, int64_t n_max, void* stream, sdr_handle** out) {
  if (!p || !out || n_max <= 0) return SDR_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->m < 1 || p->m > M_MAX || p->k < 0 || p->k > K_MAX - 1 || p->t < 1 || p->t > T_MAX) return SDR_ERR_INVALID_ARG;
  if (p->s > S_MAX || p->s < p->m + p->k + 2 || p->zeta < 1 || p->zeta > p->s || p->zeta > ZETA_MAX)
    return SDR_ERR_INVALID_ARG;
  if (!(p->rel_tol > 0.0) || !(p->safety0 >= 1.0) || p->max_cycles < 1) return SDR_ERR_INVALID_ARG;
  if (p->precision != SDR_PREC_F64 && p->precision != SDR_PREC_F32_REFINED) return SDR_ERR_INVALID_ARG;
  if (!(p->inner_rel_tol >= 0.0 && p->inner_rel_tol < 1.0)) return SDR_ERR_INVALID_ARG;
  if (n_max >= ((int64_t)1 << 31)) return SDR_ERR_INVALID_ARG;
  if (p->stale_check != 0 && p->stale_check != 1) return SDR_ERR_INVALID_ARG;
  if (p->sketch_kind != 0 && p->sketch_kind != 1) return SDR_ERR_INVALID_ARG;
  if (p->sketch_kind == 1 && n_max >= ((int64_t)1 << 29)) return SDR_ERR_INVALID_ARG;
  if (p->reserved[0] || p->reserved[1]) return SDR_ERR_INVALID_ARG;
  sdr_handle* h = new sdr_handle();
  h->p = *p;
  if (!(h->p.inner_rel_tol > 0.0)) h->p.inner_rel_tol = 1e-4;
  h->prec = p->precision;
  h->n_max = n_max;
  h->ust = (cudaStream_t)stream;
  cudaGetDevice(&h->device);
  WS& ws = h->ws;
  ws.n = n_max;
  // tall arrays: columns start on 256-byte boundaries, and a column holds at
  // least one entry past an odd n (the tensor-core recycle product copies
  // column segments of an even number of rows)
  ws.ldv = (n_max + 32) & ~(int64_t)31;
  ws.recycle_int = (p->test_flags & 4) ? 1 : 0;
  ws.sketch_kind = p->sketch_kind;
  ws.dct_n = 0;  // set by sdr_set_sketch_draws
  ws.m = p->m;
  ws.k = p->k;
  ws.t = p->t;
  ws.s = p->s;
  ws.zeta = p->zeta;
  ws.kmax = p->k + 1;
  ws.dmax = D_MAX;
  ws.seed = p->seed;
  // the sparse sign's 1/sqrt(zeta) is applied when an accumulator is read; the
  // DCT sketch scales each row as it accumulates
  ws.inv_sqrt_zeta = p->sketch_kind == 1 ? 1.0 : 1.0 / std::sqrt((double)p->zeta);
  ws.win_bits = ceil_log2(n_max) + 1;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  ws.grid_max = (nsm > 0 ? nsm : 152) * 8;  // 152 SMs on GB300, if the query fails
  const int64_t N = ws.ldv;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  // tall arrays in the storage type (8 or 4 bytes per element)
  const size_t esz = h->prec == SDR_PREC_F64 ? sizeof(double) : sizeof(float);
  auto tall = [&](void** q, size_t count) {
    unsigned char* b = nullptr;
    chk(halloc(h, &b, count * esz));
    *q = b;
  };
  // the V slab has a front column before V(:, 1): the recycle product copies
  // V(:, 0) there so that V(:, 0:m) is one 2D array
  {
    void* slab = nullptr;
    tall(&slab, (size_t)N * (p->m + 1));
    ws.Vs = slab ? (void*)((unsigned char*)slab + (size_t)N * esz) : nullptr;
  }
  tall(&ws.R[0], (size_t)N);
  tall(&ws.R[1], (size_t)N);
  tall(&ws.Wv, (size_t)N);
  tall(&ws.Xw, (size_t)N);
  tall(&ws.U[0], (size_t)N * ws.kmax);
  tall(&ws.U[1], (size_t)N * ws.kmax);
  chk(halloc(h, &h->d_tmp, (size_t)N));  // float64 scratch (A u, and the outer residual)
  if (h->prec == SDR_PREC_F32_REFINED) {
    tall(&h->rhs32, (size_t)N);
    tall(&h->dx32, (size_t)N);
  }
  chk(halloc(h, &h->st_rowptr, (size_t)N + 1));
  chk(halloc(h, &h->st_b, (size_t)N));
  chk(halloc(h, &h->st_x, (size_t)N));
  chk(cudaMallocHost((void**)&h->hc, sizeof(Ctl)));
  h->use_graphs = (p->test_flags & 2) == 0;
  const int tileR = sketch_tile_rows(p->zeta);
  const int64_t ntiles = (n_max + tileR - 1) / tileR;
  ws.ntiles = (int)ntiles;
  chk(halloc(h, &h->sk_ent, (size_t)ntiles * tileR * p->zeta));
  chk(halloc(h, &h->sk_ptr, (size_t)ntiles * PTR_STRIDE));
  ws.sk_ent = h->sk_ent;
  ws.sk_ptr = h->sk_ptr;
  chk(halloc(h, &ws.part, (size_t)ws.grid_max * 2 * NPART));
  chk(halloc(h, &ws.part2, (size_t)ws.grid_max * 2 * NPART));
  chk(halloc(h, &ws.acc, (size_t)6 * S_MAX + 16));
  chk(halloc(h, &ws.accV, CYCLE_SCRATCH_WORDS));
  ws.tctr = (int*)(ws.accV + (size_t)(M_MAX + 2) * 2 * S_MAX);
  ws.dacc = ws.accV + (size_t)(M_MAX + 2) * 2 * S_MAX + (M_MAX + 2);
  chk(halloc(h, &ws.part3, (size_t)ws.grid_max * 2 * NPART));
  chk(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
  {
    // the control stream's one-CTA kernels sit on the critical path of a cycle:
    // give them the scheduler's precedence over the streaming kernels
    int lo_pri = 0, hi_pri = 0;
    chk(cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
    chk(cudaStreamCreateWithPriority(&h->st2, cudaStreamNonBlocking, hi_pri));
  }
  chk(cudaEventCreateWithFlags(&h->evIn, cudaEventDisableTiming));
  chk(cudaEventCreateWithFlags(&h->evOut, cudaEventDisableTiming));
  chk(cudaEventCreateWithFlags(&h->evFork, cudaEventDisableTiming));
  chk(cudaEventCreateWithFlags(&h->evJoin, cudaEventDisableTiming));
  for (int j = 0; j <= M_MAX + 1 && e == cudaSuccess; ++j) {
    cudaEvent_t a = nullptr, b = nullptr;
    chk(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    if (a) h->evS.push_back(a);
    chk(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    if (b) h->evD.push_back(b);
  }
  const int s = p->s;
  chk(halloc(h, &ws.SV, (size_t)s * (M_MAX + 1)));
  chk(halloc(h, &ws.SAV, (size_t)s * M_MAX));
  for (int i = 0; i < 2; ++i) {
    chk(halloc(h, &ws.SU[i], (size_t)s * K_MAX));
    chk(halloc(h, &ws.SAU[i], (size_t)s * K_MAX));
  }
  chk(halloc(h, &ws.Y, (size_t)s * D_MAX));
  chk(halloc(h, &ws.T, (size_t)D_MAX * D_MAX));
  chk(halloc(h, &ws.Yq, (size_t)s * D_MAX));
  chk(halloc(h, &ws.Tq, (size_t)D_MAX * D_MAX));
  chk(halloc(h, &ws.texp, (size_t)D_MAX));
  chk(halloc(h, &ws.Rf, (size_t)D_MAX * D_MAX));
  chk(halloc(h, &ws.tau, (size_t)D_MAX));
  chk(halloc(h, &ws.z, (size_t)S_MAX));
  chk(halloc(h, &ws.Sr0, (size_t)S_MAX));
  chk(halloc(h, &ws.ytil, (size_t)D_MAX));
  chk(halloc(h, &ws.P, (size_t)D_MAX * K_MAX));
  chk(halloc(h, &ws.Pq, (size_t)D_MAX * K_MAX));
  chk(halloc(h, &ws.Pexp, (size_t)K_MAX));
  chk(halloc(h, &ws.ytq, (size_t)D_MAX));
  chk(halloc(h, &ws.yexp, (size_t)4));
  chk(halloc(h, &ws.dscr, ce_scratch_doubles()));
  chk(halloc(h, &ws.hist, (size_t)HIST_MAX));
  if (p->sketch_kind == 1) {
    signed char* sg = nullptr;
    int* fk = nullptr;
    double *cs = nullptr, *sc = nullptr;
    chk(halloc(h, &sg, (size_t)n_max));
    chk(halloc(h, &fk, (size_t)S_MAX));
    chk(halloc(h, &cs, (size_t)n_max + 1));
    chk(halloc(h, &sc, (size_t)S_MAX));
    ws.dct_sign = sg;
    ws.dct_k = fk;
    ws.dct_cos = cs;
    ws.dct_scale = sc;
  }
  chk(halloc(h, &ws.hist_givens, (size_t)2 * HIST_MAX));
  chk(halloc(h, &ws.log, (size_t)LOG_MAX));
  chk(halloc(h, &ws.ctl, (size_t)1));
  if (e != cudaSuccess) {
    sdr_status st = cuda_status(e);
    sdr_destroy(h);
    return st;
  }
  chk(cudaMemsetAsync(ws.acc, 0, (6 * S_MAX + 16) * sizeof(unsigned long long), h->st));
  chk(cudaMemsetAsync(ws.accV, 0, CYCLE_SCRATCH_WORDS * sizeof(unsigned long long), h->st));
  chk(cudaMemsetAsync(ws.ctl, 0, sizeof(Ctl), h->st));
  chk(cudaMemsetAsync(ws.T, 0, (size_t)D_MAX * D_MAX * sizeof(double), h->st));
  chk(cudaMemsetAsync(ws.Rf, 0, (size_t)D_MAX * D_MAX * sizeof(double), h->st));
  chk(cudaMemsetAsync(ws.P, 0, (size_t)D_MAX * K_MAX * sizeof(double), h->st));
  {
    Ctl init;
    std::memset(&init, 0, sizeof(init));
    init.safety0 = p->safety0;
    init.safety = p->safety0;
    init.persist_safety = p->persist_safety;
    init.force_svd = (p->test_flags & 1) ? 1 : 0;
    chk(cudaMemcpyAsync(ws.ctl, &init, sizeof(Ctl), cudaMemcpyHostToDevice, h->st));
  }
  chk(launch_sketch_build(ws, n_max, h->sk_ent, h->sk_ptr, h->st));
  chk(cudaStreamSynchronize(h->st));
  if (e != cudaSuccess) {
    sdr_status st = cuda_status(e);
    sdr_destroy(h);
    return st;
  }
  *out = h;
  return SDR_OK;
}

}  // extern "C"

namespace {

// State of a run of restart cycles (one sdr_solve of the float64 solver, or
// one inner solve of the refined form), advanced one cycle at a time so that
// a batch of handles can be driven in lockstep.
template <typename T>
struct CycleRun {
  sdr_handle* h = nullptr;
  WS ws;
  CsrDev Ad;
  const T* b = nullptr;
  T* x = nullptr;
  T* xcur = nullptr;
  T* xoth = nullptr;
  int rb = 0;
  int max_cycles = 0;
  int cycles = 0, full_svd = 0;
  bool converged = false, active = false;
  sdr_status status = SDR_OK;
  Ctl hc;  // control block after the last completed cycle
};

// One cycle's launches (Algorithm 1): the Arnoldi kernels on st, the dense
// step and the true-residual check of each column on st2, the cycle end on st.
// Two streams per cycle: the dense step of column j-1 needs step j's SpMV
// (which sketches and finishes column j); step j waits for the control work
// of column j - SPEC_LAG, so it knows whether an earlier check ended the cycle.
template <typename T>
sdr_status issue_cycle(sdr_handle* h, const WS& ws, const CsrDev& Ad, const T* b, T* xcur, T* xoth, int rb,
                       int cu, int kh) {
  cudaStream_t st = h->st, st2 = h->st2;
  const int m = ws.m;
  unsigned long long* accR = ws.acc + 2 * S_MAX;
  const T* vcol[M_MAX + 1];
  vcol[0] = (const T*)ws.R[rb];
  for (int c = 1; c <= m; ++c) vcol[c] = tall_col<T>(ws.Vs, ws.ldv, c - 1);
  const T* Ucur = (const T*)ws.U[cu];
  SDR_CK(cudaMemsetAsync(ws.accV, 0, CYCLE_SCRATCH_WORDS * sizeof(unsigned long long), st));
  SDR_LAUNCH(h, SDR_K_CYCLE_INIT, launch_cycle_head(ws, kh, accR, h->p.persist_safety, st));
  SDR_CK(cudaEventRecord(h->evFork, st));
  SDR_CK(cudaStreamWaitEvent(st2, h->evFork, 0));
  SDR_LAUNCH_ON(h, SDR_K_CYCLE_INIT, st2, launch_cycle_qr(ws, ws.SAU[cu], kh, st2));
  for (int j = 0; j <= m; ++j) {
    if (j >= SPEC_LAG) SDR_CK(cudaStreamWaitEvent(st, h->evD[j - SPEC_LAG], 0));
    if (j < m) {
      if (ws.sketch_kind && j >= 1)  // the DCT sketch of v_hat_j (the sparse sign is fused into the SpMV)
        SDR_LAUNCH(h, SDR_K_SKETCH,
                   launch_sketch_vec<T>(ws, vcol[j], ws.n, ws.accV + (int64_t)j * 2 * S_MAX,
                                        ctl_int_field(ws.ctl, offsetof(Ctl, vtop) + j * sizeof(int)), st));
      SDR_LAUNCH(h, SDR_K_SPMV_DOTS, launch_spmv_dots<T>(ws, Ad, vcol, j, st));
    } else {
      SDR_LAUNCH(h, SDR_K_SKETCH, launch_sketch_col<T>(ws, vcol[m], m, st));
    }
    if (j >= 1) {
      SDR_CK(cudaEventRecord(h->evS[j], st));
      SDR_CK(cudaStreamWaitEvent(st2, h->evS[j], 0));
      SDR_LAUNCH_ON(h, SDR_K_STEP_DENSE, st2, launch_step_dense(ws, j - 1, kh, cu, accR, st2));
      SDR_LAUNCH_ON(h, SDR_K_CHECK_GEMV, st2, launch_check_gemv<T>(ws, Ucur, vcol, xcur, xoth, kh, j - 1, cu, st2));
      SDR_LAUNCH_ON(h, SDR_K_CHECK_RESIDUAL, st2,
                    launch_residual<T>(ws, Ad, b, xoth, (T*)ws.R[1 - rb], accR, j - 1, 1, st2));
      SDR_CK(cudaEventRecord(h->evD[j - 1], st2));
    }
    if (j < m) SDR_LAUNCH(h, SDR_K_UPDATE_SKETCH, launch_update_sketch<T>(ws, vcol, (T*)vcol[j + 1], j, st));
  }
  SDR_CK(cudaEventRecord(h->evJoin, st2));
  SDR_CK(cudaStreamWaitEvent(st, h->evJoin, 0));
  for (int part = 0; part < CYCLE_END_PARTS; ++part)
    SDR_LAUNCH(h, part == 0 ? SDR_K_CYCLE_END : SDR_K_CE_RINV + part - 1,
               launch_cycle_end_part(part, ws, kh, cu, ws.SU[cu], ws.SAU[cu], ws.SU[1 - cu], ws.SAU[1 - cu], st));
  SDR_LAUNCH(h, SDR_K_RECYCLE_GEMM, launch_recycle_gemm<T>(ws, Ucur, vcol, (T*)ws.U[1 - cu], kh, cu, 1 - cu, st));
  return SDR_OK;
}

// Issue one cycle, through a cached CUDA graph when the handle uses graphs
// and per-launch profiling is off.
template <typename T>
sdr_status launch_cycle(CycleRun<T>& r) {
  sdr_handle* h = r.h;
  const int cu = h->cu, kh = h->kh;
  const int xpar = r.xcur == r.x ? 0 : 1;
  if (!h->use_graphs || h->prof.on) return issue_cycle<T>(h, r.ws, r.Ad, r.b, r.xcur, r.xoth, r.rb, cu, kh);
  for (auto& g : h->graphs) {
    if (g.n == r.Ad.n && g.nnz == r.Ad.nnz && g.kh == kh && g.cu == cu && g.rb == r.rb && g.xpar == xpar) {
      h->launches += g.kernels;
      return cuda_status(cudaGraphLaunch(g.exec, h->st));
    }
  }
  const int before = h->launches;
  SDR_CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  const sdr_status s1 = issue_cycle<T>(h, r.ws, r.Ad, r.b, r.xcur, r.xoth, r.rb, cu, kh);
  cudaGraph_t graph = nullptr;
  const cudaError_t e1 = cudaStreamEndCapture(h->st, &graph);
  if (s1 != SDR_OK || e1 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return s1 != SDR_OK ? s1 : cuda_status(e1);
  }
  // the kernels keep the priority of the stream they were captured on (the
  // control stream's dense steps ahead of the SpMV's CTAs), as in direct launches
  cudaGraphExec_t exec = nullptr;
  cudaError_t e2 = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  if (e2 != cudaSuccess) {
    (void)cudaGetLastError();
    e2 = cudaGraphInstantiate(&exec, graph, 0);
  }
  cudaGraphDestroy(graph);
  SDR_CK(e2);
  sdr_handle::GraphEntry g{r.Ad.n, r.Ad.nnz, kh, cu, r.rb, xpar, h->launches - before, exec};
  h->graphs.push_back(g);
  return cuda_status(cudaGraphLaunch(exec, h->st));
}

// Solve start: ||b||, tol, r0 = b - A x with S r0; the control block is
// copied to the pinned host copy (read by run_complete_init).
template <typename T>
sdr_status run_begin(CycleRun<T>& r, sdr_handle* h, const CsrDev& Ad, const T* b, T* x, double rel_tol,
                     int max_cycles, bool keep_logs = false) {
  r.h = h;
  r.ws = h->ws;
  r.ws.n = Ad.n;
  r.Ad = Ad;
  r.b = b;
  r.x = x;
  r.xcur = x;
  r.xoth = (T*)r.ws.Xw;
  r.rb = 0;
  r.max_cycles = max_cycles;
  r.active = false;
  r.converged = false;
  r.status = SDR_OK;
  unsigned long long* accR = r.ws.acc + 2 * S_MAX;
  SDR_LAUNCH(h, SDR_K_SOLVE_INIT, launch_solve_init_x<T>(r.ws, Ad, b, x, rel_tol, h->st, keep_logs));
  SDR_LAUNCH(h, SDR_K_RESIDUAL0, launch_residual<T>(r.ws, Ad, b, x, (T*)r.ws.R[0], accR, -1, 0, h->st));
  SDR_CK(cudaMemcpyAsync(h->hc, r.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st));
  return SDR_OK;
}

template <typename T>
sdr_status run_complete_init(CycleRun<T>& r) {
  SDR_CK(cudaStreamSynchronize(r.h->st));
  r.hc = *r.h->hc;
  r.converged = r.hc.converged != 0;
  // a NaN or an Inf in b, x0 or A shows in ||b||, ||A||_inf or ||b - A x0||:
  // no cycle is issued and the solve ends with SDR_ERR_BREAKDOWN, x unchanged
  if (!std::isfinite(r.hc.bnorm) || !std::isfinite(r.hc.anorm_inf) || !std::isfinite(r.hc.res)) {
    r.converged = false;
    r.status = SDR_ERR_BREAKDOWN;
  }
  r.active = !r.converged && r.status == SDR_OK && r.cycles < r.max_cycles;
  return SDR_OK;
}

template <typename T>
sdr_status run_issue(CycleRun<T>& r) {
  const sdr_status s = launch_cycle<T>(r);
  if (s != SDR_OK) return s;
  SDR_CK(cudaMemcpyAsync(r.h->hc, r.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, r.h->st));
  return SDR_OK;
}

// Read the cycle's outcome and advance the host state (buffer parities,
// recycle dimension, convergence).
template <typename T>
sdr_status run_complete(CycleRun<T>& r) {
  sdr_handle* h = r.h;
  SDR_CK(cudaStreamSynchronize(h->st));
  r.hc = *h->hc;
  const Ctl& hc = r.hc;
  ++r.cycles;
  if (hc.jf > 0) {
    h->cu = 1 - h->cu;
    h->kh = hc.kprime;
    T* t = r.xcur;
    r.xcur = r.xoth;
    r.xoth = t;
    r.rb = 1 - r.rb;
    if (hc.svd_path) ++r.full_svd;
  }
  r.converged = hc.converged != 0;
  if (!r.converged && (hc.bd_dense || !std::isfinite(hc.res))) r.status = SDR_ERR_BREAKDOWN;
  if (hc.tc_error) r.status = SDR_ERR_CUDA;  // a bounded wait of the recycle product ran out
  r.active = !r.converged && r.status == SDR_OK && r.cycles < r.max_cycles;
  return SDR_OK;
}

template <typename T>
sdr_status run_finish(CycleRun<T>& r) {
  if (r.xcur != r.x)
    SDR_CK(cudaMemcpyAsync(r.x, r.xcur, (size_t)r.Ad.n * sizeof(T), cudaMemcpyDeviceToDevice, r.h->st));
  if (r.status == SDR_OK && !r.converged) r.status = SDR_ERR_NOT_CONVERGED;
  return SDR_OK;
}

// Restarted GMRES-SDR on A x = b with tall vectors of type T, from the
// iterate in x, for at most max_cycles cycles; x is overwritten with the
// result.  tol = rel_tol ||b||.
template <typename T>
sdr_status run_cycles(sdr_handle* h, const CsrDev& Ad, const T* b, T* x, double rel_tol, int max_cycles,
                      CycleRun<T>& r, bool keep_logs = false) {
  sdr_status s = run_begin<T>(r, h, Ad, b, x, rel_tol, max_cycles, keep_logs);
  if (s == SDR_OK) s = run_complete_init<T>(r);
  while (s == SDR_OK && r.active) {
    s = run_issue<T>(r);
    if (s == SDR_OK) s = run_complete<T>(r);
  }
  if (s == SDR_OK) s = run_finish<T>(r);
  return s;
}

// Copy the caller's matrix into the handle's staging buffers (graphs are
// captured against them).  Reallocates when nnz grows.
sdr_status stage_matrix(sdr_handle* h, const sdr_csr* A, CsrDev& out) {
  if (A->nnz > h->st_nnz_cap) {
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    cudaFree(h->st_col);
    cudaFree(h->st_val);
    cudaFree(h->st_val32);
    h->st_col = nullptr;
    h->st_val = nullptr;
    h->st_val32 = nullptr;
    h->st_nnz_cap = 0;
    const size_t cap = (size_t)(A->nnz > 0 ? A->nnz : 1);
    SDR_CK(cudaMalloc(&h->st_col, cap * sizeof(int32_t)));
    SDR_CK(cudaMalloc(&h->st_val, cap * sizeof(double)));
    if (h->prec == SDR_PREC_F32_REFINED) SDR_CK(cudaMalloc(&h->st_val32, cap * sizeof(float)));
    h->st_nnz_cap = (int64_t)cap;
  }
  cudaStream_t st = h->st;
  SDR_CK(cudaMemcpyAsync(h->st_rowptr, A->rowptr, (size_t)(A->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  if (A->nnz > 0) {
    SDR_CK(cudaMemcpyAsync(h->st_col, A->col, (size_t)A->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    SDR_CK(cudaMemcpyAsync(h->st_val, A->val, (size_t)A->nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (h->prec == SDR_PREC_F32_REFINED)
      SDR_CK(cudaMemcpyAsync(h->st_val32, A->val32, (size_t)A->nnz * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  out = CsrDev{A->n, A->nnz, h->st_rowptr, h->st_col, h->st_val, h->st_val32};
  return SDR_OK;
}

// Per-solve bookkeeping shared by sdr_solve and sdr_solve_batch.
struct SolveCtx {
  CycleRun<double> run;
  CsrDev Ad;
  const double* b = nullptr;
  double* x = nullptr;       // the iterate the cycles work on (staging or the caller's)
  double* x_user = nullptr;  // the caller's x
};

sdr_status solve_begin_f64(sdr_handle* h, const sdr_csr* A, const double* b, double* x, SolveCtx& c) {
  cudaStream_t st = h->st;
  h->launches = 0;
  h->sau_refreshes = 0;
  h->extra_matvecs = 0;
  // anything a failed earlier call left on the control stream comes first
  SDR_CK(cudaEventRecord(h->evJoin, h->st2));
  SDR_CK(cudaStreamWaitEvent(st, h->evJoin, 0));
  c.x_user = x;
  if (h->use_graphs && !h->prof.on) {
    const sdr_status s = stage_matrix(h, A, c.Ad);
    if (s != SDR_OK) return s;
    SDR_CK(cudaMemcpyAsync(h->st_b, b, (size_t)A->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SDR_CK(cudaMemcpyAsync(h->st_x, x, (size_t)A->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    c.b = h->st_b;
    c.x = h->st_x;
  } else {
    c.Ad = to_dev(A);
    c.b = b;
    c.x = x;
  }
  return run_begin<double>(c.run, h, c.Ad, c.b, c.x, h->p.rel_tol, h->p.max_cycles);
}

sdr_status solve_end(sdr_handle* h, const CycleRun<double>* run_f64, const Ctl& hc, int cycles, int full_svd,
                     bool converged, int refinements, double final_res, double bnorm, double tol,
                     sdr_stats* stats) {
  (void)run_f64;
  cudaStream_t st = h->st;
  const WS& ws = h->ws;
  const int nh = hc.hist_n < HIST_MAX ? hc.hist_n : HIST_MAX;
  const int nl = hc.log_n < LOG_MAX ? hc.log_n : LOG_MAX;
  h->hist.assign(nh, 0.0);
  h->log.assign(nl, CycleLog());
  if (nh) SDR_CK(cudaMemcpyAsync(h->hist.data(), ws.hist, nh * sizeof(double), cudaMemcpyDeviceToHost, st));
  h->hist_givens.assign(2 * (size_t)nh, 0.0);
  if (nh)
    SDR_CK(cudaMemcpyAsync(h->hist_givens.data(), ws.hist_givens, 2 * nh * sizeof(double), cudaMemcpyDeviceToHost,
                           st));
  if (nl) SDR_CK(cudaMemcpyAsync(h->log.data(), ws.log, nl * sizeof(CycleLog), cudaMemcpyDeviceToHost, st));
  SDR_CK(cudaStreamSynchronize(st));
  SDR_CK(prof_collect(h));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->cycles = cycles;
    stats->converged = converged ? 1 : 0;
    stats->matvecs = hc.matvecs;
    stats->sketches = hc.sketches;
    int checks = 0;
    for (auto& g : h->log) checks += g.checks;
    stats->true_res_evals = checks;
    stats->arnoldi_steps = hc.hist_n;
    stats->recycle_dim = h->kh;
    stats->full_svd_cycles = full_svd;
    stats->kernel_launches = h->launches;
    stats->refinements = refinements;
    stats->sau_refreshes = h->sau_refreshes;
    stats->refresh_matvecs = h->extra_matvecs;
    stats->matvecs += h->extra_matvecs;
    stats->final_res = final_res;
    stats->tol = tol;
    stats->bnorm = bnorm;
    stats->final_rel_res = bnorm > 0.0 ? final_res / bnorm : final_res;
  }
  return SDR_OK;
}

sdr_status solve_finish_f64(sdr_handle* h, SolveCtx& c, sdr_stats* stats) {
  SDR_CK(cudaGetLastError());
  sdr_status s = run_finish<double>(c.run);
  if (s != SDR_OK) return s;
  if (c.x != c.x_user)
    SDR_CK(cudaMemcpyAsync(c.x_user, c.x, (size_t)c.Ad.n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  const Ctl& hc = c.run.hc;
  s = solve_end(h, &c.run, hc, c.run.cycles, c.run.full_svd, c.run.converged, 0, hc.res, hc.bnorm, hc.tol, stats);
  return s != SDR_OK ? s : c.run.status;
}

}  // namespace

extern "C" {

sdr_status sdr_solve(sdr_handle* h, const sdr_csr* A, const double* b, double* x, sdr_stats* stats) {
  if (!h || !csr_ok(h, A) || !b || !x) return SDR_ERR_INVALID_ARG;
  StreamGuard guard(h);
  h->sau_refreshes = 0;
  h->extra_matvecs = 0;
  if (h->prec == SDR_PREC_F64) {
    SolveCtx c;
    sdr_status s = solve_begin_f64(h, A, b, x, c);
    if (s == SDR_OK) s = run_complete_init<double>(c.run);
    while (s == SDR_OK && c.run.active) {
      s = run_issue<double>(c.run);
      if (s == SDR_OK) s = run_complete<double>(c.run);
      // stale_check: a cycle whose last true residual exceeds 4 sres had a stale
      // SAU; recompute it for the new recycle space before the next cycle
      const Ctl& hc = c.run.hc;
      if (s == SDR_OK && c.run.active && h->p.stale_check && h->kh > 0 && hc.res > 4.0 * hc.sres) {
        const sdr_csr cur{c.Ad.n, c.Ad.nnz, c.Ad.rowptr, c.Ad.col, c.Ad.val, c.Ad.val32};
        const int l0 = h->launches;
        s = issue_sau<double>(h, &cur, c.Ad.n);
        h->launches += l0;
        ++h->sau_refreshes;
        h->extra_matvecs += h->kh;
      }
    }
    if (s != SDR_OK) return s;
    return solve_finish_f64(h, c, stats);
  }
  // Iterative refinement in float64 around the float32 solver: the outer
  // residual r = b - A x uses the float64 values; each inner solve of
  // A d = r runs with float32 storage and arithmetic and keeps the recycle
  // space (same matrix, new right-hand side: Section 3.6).
  WS ws = h->ws;
  ws.n = A->n;
  cudaStream_t st = h->st;
  h->launches = 0;
  SDR_CK(cudaEventRecord(h->evJoin, h->st2));
  SDR_CK(cudaStreamWaitEvent(st, h->evJoin, 0));
  CsrDev Ad;
  if (h->use_graphs && !h->prof.on) {
    const sdr_status s = stage_matrix(h, A, Ad);
    if (s != SDR_OK) return s;
  } else {
    Ad = to_dev(A);
  }
  unsigned long long* accR = ws.acc + 2 * S_MAX;
  double* r64 = h->d_tmp;
  SDR_LAUNCH(h, SDR_K_SOLVE_INIT, launch_solve_init_x<double>(ws, Ad, b, x, h->p.rel_tol, st));
  SDR_CK(cudaMemcpyAsync(h->hc, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  SDR_CK(cudaStreamSynchronize(st));
  const double bnorm = h->hc->bnorm, tol = h->hc->tol;
  const int max_refine = 40;
  bool conv = false;
  sdr_status status = SDR_OK;
  double last_res = INFINITY, final_res = 0.0;
  int refinements = 0, cycles = 0, full_svd = 0;
  CycleRun<float> run;
  for (;;) {
    SDR_LAUNCH(h, SDR_K_RESIDUAL0, launch_residual<double>(ws, Ad, b, x, r64, accR, -1, 0, st));
    SDR_CK(cudaMemsetAsync(accR, 0, 2 * S_MAX * sizeof(unsigned long long), st));
    SDR_CK(cudaMemcpyAsync(h->hc, ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    SDR_CK(cudaStreamSynchronize(st));
    final_res = h->hc->res;
    if (!std::isfinite(final_res)) {
      status = SDR_ERR_BREAKDOWN;
      break;
    }
    if (final_res < tol) {
      conv = true;
      break;
    }
    // stop when refinement no longer reduces the residual
    if (refinements >= max_refine || (refinements > 0 && !(final_res < 0.5 * last_res))) break;
    last_res = final_res;
    SDR_LAUNCH(h, SDR_K_REFINE, launch_to_f32(r64, (float*)h->rhs32, (float*)h->dx32, Ad.n, st));
    run = CycleRun<float>();
    const sdr_status rs = run_cycles<float>(h, Ad, (const float*)h->rhs32, (float*)h->dx32, h->p.inner_rel_tol,
                                            h->p.max_cycles, run, /*keep_logs=*/true);
    if (rs != SDR_OK) return rs;
    cycles += run.cycles;
    full_svd += run.full_svd;
    if (run.status == SDR_ERR_BREAKDOWN || run.status == SDR_ERR_RANK) {
      status = run.status;
      break;
    }
    SDR_LAUNCH(h, SDR_K_REFINE, launch_add_f32(x, (const float*)h->dx32, Ad.n, st));
    ++refinements;
  }
  if (status == SDR_OK && !conv) status = SDR_ERR_NOT_CONVERGED;
  const sdr_status s = solve_end(h, nullptr, run.hc, cycles, full_svd, conv, refinements, final_res, bnorm, tol,
                                 stats);
  return s != SDR_OK ? s : status;
}

sdr_status sdr_solve_batch(int32_t count, sdr_handle* const* hs, const sdr_csr* As, const double* const* bs,
                           double* const* xs, sdr_stats* stats) {
  if (count < 0 || (count > 0 && (!hs || !As || !bs || !xs))) return SDR_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !csr_ok(hs[i], &As[i]) || !bs[i] || !xs[i]) return SDR_ERR_INVALID_ARG;
    if (hs[i]->prec != SDR_PREC_F64) return SDR_ERR_NOT_IMPLEMENTED;
    for (int q = 0; q < i; ++q)
      if (hs[q] == hs[i]) return SDR_ERR_INVALID_ARG;
  }
  std::vector<std::unique_ptr<StreamGuard>> guards;
  for (int i = 0; i < count; ++i) guards.emplace_back(new StreamGuard(hs[i]));
  std::vector<SolveCtx> ctx(count);
  for (int i = 0; i < count; ++i) {
    const sdr_status s = solve_begin_f64(hs[i], &As[i], bs[i], xs[i], ctx[i]);
    if (s != SDR_OK) return s;
  }
  for (int i = 0; i < count; ++i) {
    const sdr_status s = run_complete_init<double>(ctx[i].run);
    if (s != SDR_OK) return s;
  }
  // Lockstep rounds: one cycle of every unfinished system is issued (each on
  // its handle's streams, so the systems' kernels run concurrently), then
  // every issued cycle is completed.
  for (;;) {
    bool any = false;
    for (int i = 0; i < count; ++i) {
      if (!ctx[i].run.active) continue;
      any = true;
      const sdr_status s = run_issue<double>(ctx[i].run);
      if (s != SDR_OK) return s;
    }
    if (!any) break;
    for (int i = 0; i < count; ++i) {
      if (!ctx[i].run.active) continue;
      const sdr_status s = run_complete<double>(ctx[i].run);
      if (s != SDR_OK) return s;
    }
  }
  sdr_status worst = SDR_OK;
  for (int i = 0; i < count; ++i) {
    const sdr_status s = solve_finish_f64(hs[i], ctx[i], stats ? &stats[i] : nullptr);
    if (s == SDR_ERR_CUDA) return s;
    if (s != SDR_OK && worst == SDR_OK) worst = s;
  }
  return worst;
}

sdr_status sdr_recycle_batch(int32_t count, sdr_handle* const* hs, const sdr_csr* As, int32_t mode) {
  if (count < 0 || (count > 0 && (!hs || (mode == 0 && !As)))) return SDR_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return SDR_ERR_INVALID_ARG;
    if (mode == 0 && hs[i]->kh > 0 && !csr_ok(hs[i], &As[i])) return SDR_ERR_INVALID_ARG;
  }
  std::vector<std::unique_ptr<StreamGuard>> guards;
  for (int i = 0; i < count; ++i) guards.emplace_back(new StreamGuard(hs[i]));
  for (int i = 0; i < count; ++i) {
    sdr_handle* h = hs[i];
    if (mode == 2) {
      h->kh = 0;
    } else if (mode == 0 && h->kh > 0) {
      const sdr_status s = h->prec == SDR_PREC_F64 ? issue_sau<double>(h, &As[i], As[i].n)
                                                   : issue_sau<float>(h, &As[i], As[i].n);
      if (s != SDR_OK) return s;
    } else if (mode != 1 && mode != 0) {
      return SDR_ERR_INVALID_ARG;
    }
  }
  sdr_status worst = SDR_OK;
  for (int i = 0; i < count; ++i) {
    SDR_CK(cudaStreamSynchronize(hs[i]->st));
    SDR_CK(prof_collect(hs[i]));
    if (mode == 0) {
      const sdr_status s = verify_sau_rank(hs[i]);
      if (s == SDR_ERR_CUDA) return s;
      if (s != SDR_OK && worst == SDR_OK) worst = s;
    }
  }
  return worst;
}

}  // extern "C"

// Recompute SAU = S A U column by column (exact variant, Section 3.6);
// issue_sau only enqueues the work on the handle's stream.
template <typename T>
static sdr_status issue_sau(sdr_handle* h, const sdr_csr* A, int64_t n) {
  WS ws = h->ws;
  ws.n = n;
  const CsrDev Ad = to_dev(A);
  unsigned long long* accG = ws.acc + 4 * S_MAX;
  int* topG = ctl_int_field(ws.ctl, offsetof(Ctl, accG_top));
  h->launches = 0;
  for (int c = 0; c < h->kh; ++c) {
    const T* u = tall_col<T>(ws.U[h->cu], ws.ldv, c);
    T* au = (T*)h->d_tmp;
    SDR_CK(prof_begin(h, SDR_K_RECYCLE_SAU, h->st));
    SDR_CK(launch_spmv<T>(Ad, u, au, h->st));
    SDR_CK(launch_maxabs_top<T>(ws, au, n, topG, h->st));
    SDR_CK(launch_sketch_vec<T>(ws, au, n, accG, topG, h->st));
    SDR_CK(launch_sketch_finish(ws, accG, topG, ws.SAU[h->cu] + (int64_t)c * ws.s, h->st));
    SDR_CK(prof_end(h, h->st));
  }
  return SDR_OK;
}

template <typename T>
static sdr_status recompute_sau(sdr_handle* h, const sdr_csr* A, int64_t n) {
  const sdr_status s = issue_sau<T>(h, A, n);
  if (s != SDR_OK) return s;
  SDR_CK(cudaStreamSynchronize(h->st));
  SDR_CK(prof_collect(h));
  return SDR_OK;
}

template <typename T>
static sdr_status recompute_su(sdr_handle* h, int64_t n) {
  WS ws = h->ws;
  ws.n = n;
  unsigned long long* accG = ws.acc + 4 * S_MAX;
  int* topG = ctl_int_field(ws.ctl, offsetof(Ctl, accG_top));
  for (int c = 0; c < h->kh; ++c) {
    const T* u = tall_col<T>(ws.U[h->cu], ws.ldv, c);
    SDR_CK(prof_begin(h, SDR_K_SKETCH, h->st));
    h->launches += 2;  // three kernels under one timing bracket
    SDR_CK(launch_maxabs_top<T>(ws, u, n, topG, h->st));
    SDR_CK(launch_sketch_vec<T>(ws, u, n, accG, topG, h->st));
    SDR_CK(launch_sketch_finish(ws, accG, topG, ws.SU[h->cu] + (int64_t)c * ws.s, h->st));
    SDR_CK(prof_end(h, h->st));
  }
  SDR_CK(cudaStreamSynchronize(h->st));
  SDR_CK(prof_collect(h));
  return SDR_OK;
}

// After a recycle space is installed (exact recompute or import): test SAU's
// numerical column rank.  A rank-deficient SAU leaves R^{-1} of Algorithm 1's
// least squares undefined, so the space is dropped and SDR_ERR_RANK returned.
static sdr_status verify_sau_rank(sdr_handle* h) {
  if (h->kh == 0) return SDR_OK;
  int* flag = ctl_int_field(h->ws.ctl, offsetof(Ctl, rank_sau));
  SDR_CK(launch_sau_rank(h->ws.SAU[h->cu], h->ws.s, h->kh, flag, h->st));
  int hflag = 0;
  SDR_CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  SDR_CK(cudaStreamSynchronize(h->st));
  if (hflag) {
    h->kh = 0;
    return SDR_ERR_RANK;
  }
  return SDR_OK;
}

extern "C" {

sdr_status sdr_recycle(sdr_handle* h, const sdr_csr* A_next, int32_t mode) {
  if (!h) return SDR_ERR_INVALID_ARG;
  StreamGuard guard(h);
  if (mode == 2) {
    h->kh = 0;
    return SDR_OK;
  }
  if (mode == 1) return SDR_OK;
  if (mode != 0) return SDR_ERR_INVALID_ARG;
  if (h->kh == 0) return SDR_OK;
  if (!csr_ok(h, A_next)) return SDR_ERR_INVALID_ARG;
  const sdr_status s = h->prec == SDR_PREC_F64 ? recompute_sau<double>(h, A_next, A_next->n)
                                               : recompute_sau<float>(h, A_next, A_next->n);
  return s != SDR_OK ? s : verify_sau_rank(h);
}

sdr_status sdr_sketch(sdr_handle* h, const double* x, int64_t n, double* y) {
  if (!h || !x || !y || n <= 0 || n > h->n_max) return SDR_ERR_INVALID_ARG;
  if (h->ws.sketch_kind && n != h->ws.dct_n) return SDR_ERR_INVALID_ARG;
  StreamGuard guard(h);
  WS ws = h->ws;
  ws.n = n;
  unsigned long long* accG = ws.acc + 4 * S_MAX;
  int* topG = ctl_int_field(ws.ctl, offsetof(Ctl, accG_top));
  h->launches = 0;
  SDR_CK(prof_begin(h, SDR_K_SKETCH, h->st));
  h->launches += 2;  // three kernels under one timing bracket
  SDR_CK(launch_maxabs_top<double>(ws, x, n, topG, h->st));
  SDR_CK(launch_sketch_vec<double>(ws, x, n, accG, topG, h->st));
  SDR_CK(launch_sketch_finish(ws, accG, topG, y, h->st));
  SDR_CK(prof_end(h, h->st));
  SDR_CK(cudaStreamSynchronize(h->st));
  SDR_CK(prof_collect(h));
  return SDR_OK;
}

sdr_status sdr_get_history(sdr_handle* h, double* sres, int32_t cap_steps, int32_t* n_steps, sdr_cycle_log* log,
                           int32_t cap_cycles, int32_t* n_cycles) {
  if (!h) return SDR_ERR_INVALID_ARG;
  static_assert(sizeof(sdr_cycle_log) == sizeof(CycleLog), "cycle log layout");
  const int nh = (int)h->hist.size(), nl = (int)h->log.size();
  if (n_steps) *n_steps = nh;
  if (n_cycles) *n_cycles = nl;
  if (sres && cap_steps > 0) std::memcpy(sres, h->hist.data(), sizeof(double) * (nh < cap_steps ? nh : cap_steps));
  if (log && cap_cycles > 0) std::memcpy(log, h->log.data(), sizeof(CycleLog) * (nl < cap_cycles ? nl : cap_cycles));
  return SDR_OK;
}

sdr_status sdr_set_sketch_draws(sdr_handle* h, int64_t n, const int8_t* signs, const int32_t* rows) {
  if (!h || h->ws.sketch_kind != 1 || n < 1 || n > h->n_max || !signs || !rows) return SDR_ERR_INVALID_ARG;
  const int s = h->ws.s;
  for (int i = 0; i < s; ++i)
    if (rows[i] < 0 || rows[i] >= n || (i > 0 && rows[i] <= rows[i - 1])) return SDR_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (signs[i] != 1 && signs[i] != -1) return SDR_ERR_INVALID_ARG;
  StreamGuard guard(h);
  std::vector<double> scale(s);
  for (int i = 0; i < s; ++i) scale[i] = (rows[i] == 0 ? 1.0 : std::sqrt(2.0)) / std::sqrt((double)s);
  WS& ws = h->ws;
  SDR_CK(cudaMemcpyAsync((void*)ws.dct_sign, signs, (size_t)n, cudaMemcpyHostToDevice, h->st));
  SDR_CK(cudaMemcpyAsync((void*)ws.dct_k, rows, (size_t)s * sizeof(int), cudaMemcpyHostToDevice, h->st));
  SDR_CK(cudaMemcpyAsync((void*)ws.dct_scale, scale.data(), (size_t)s * sizeof(double), cudaMemcpyHostToDevice,
                         h->st));
  SDR_CK(launch_dct_table((double*)ws.dct_cos, n, h->st));
  SDR_CK(cudaStreamSynchronize(h->st));
  if (ws.dct_n != n) {  // graphs captured with another size are stale
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
  }
  ws.dct_n = n;
  h->kh = 0;  // a recycle space sketched with another operator is dropped
  return SDR_OK;
}

sdr_status sdr_get_givens(sdr_handle* h, double* sines, double* cosines, int32_t cap, int32_t* n_steps) {
  if (!h || cap < 0) return SDR_ERR_INVALID_ARG;
  const int nh = (int)(h->hist_givens.size() / 2);
  if (n_steps) *n_steps = nh;
  for (int i = 0; i < nh && i < cap; ++i) {
    if (sines) sines[i] = h->hist_givens[2 * (size_t)i];
    if (cosines) cosines[i] = h->hist_givens[2 * (size_t)i + 1];
  }
  return SDR_OK;
}

sdr_status sdr_profile(sdr_handle* h, int32_t enable) {
  if (!h) return SDR_ERR_INVALID_ARG;
  Prof& P = h->prof;
  P.on = enable != 0;
  P.cls.clear();
  P.strm.clear();
  for (int i = 0; i < SDR_K_COUNT; ++i) {
    P.total_ms[i] = 0.0;
    P.launches[i] = 0;
  }
  return SDR_OK;
}

sdr_status sdr_profile_get(sdr_handle* h, sdr_kernel_time* out, int32_t cap, int32_t* n) {
  if (!h) return SDR_ERR_INVALID_ARG;
  if (n) *n = SDR_K_COUNT;
  for (int i = 0; i < SDR_K_COUNT && i < cap && out; ++i) {
    out[i].launches = h->prof.launches[i];
    out[i].pad = 0;
    out[i].total_ms = h->prof.total_ms[i];
  }
  return SDR_OK;
}

sdr_status sdr_trace(sdr_handle* h, int32_t cap) {
  if (!h || cap < 0) return SDR_ERR_INVALID_ARG;
  Prof& P = h->prof;
  if (cap > 0 && !P.ref && cudaEventCreate(&P.ref) != cudaSuccess) return SDR_ERR_CUDA;
  P.trace_cap = cap;
  P.ref_set = false;
  P.trace.clear();
  return SDR_OK;
}

sdr_status sdr_trace_get(sdr_handle* h, sdr_trace_entry* out, int32_t cap, int32_t* n) {
  if (!h || cap < 0 || (cap > 0 && !out)) return SDR_ERR_INVALID_ARG;
  const int32_t nt = (int32_t)h->prof.trace.size();
  if (n) *n = nt;
  if (cap > 0) std::memcpy(out, h->prof.trace.data(), sizeof(sdr_trace_entry) * (size_t)(nt < cap ? nt : cap));
  return SDR_OK;
}

sdr_status sdr_recycle_dim(sdr_handle* h, int32_t* kdim) {
  if (!h || !kdim) return SDR_ERR_INVALID_ARG;
  *kdim = h->kh;
  return SDR_OK;
}

sdr_status sdr_recycle_export(sdr_handle* h, int64_t n, double* U, double* SU, double* SAU) {
  if (!h || n <= 0 || n > h->n_max) return SDR_ERR_INVALID_ARG;
  if (h->prec != SDR_PREC_F64) return SDR_ERR_NOT_IMPLEMENTED;
  StreamGuard guard(h);
  const WS& ws = h->ws;
  const int kh = h->kh;
  if (kh == 0) return SDR_OK;
  if (U)
    SDR_CK(cudaMemcpy2DAsync(U, n * sizeof(double), ws.U[h->cu], ws.ldv * sizeof(double), n * sizeof(double), kh,
                             cudaMemcpyDeviceToDevice, h->st));
  if (SU)
    SDR_CK(cudaMemcpyAsync(SU, ws.SU[h->cu], (size_t)ws.s * kh * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  if (SAU)
    SDR_CK(cudaMemcpyAsync(SAU, ws.SAU[h->cu], (size_t)ws.s * kh * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  SDR_CK(cudaStreamSynchronize(h->st));
  return SDR_OK;
}

sdr_status sdr_recycle_import(sdr_handle* h, const sdr_csr* A, int64_t n, int32_t kdim, const double* U,
                              const double* SU, const double* SAU) {
  if (!h || n <= 0 || n > h->n_max || kdim < 0 || kdim > h->ws.kmax) return SDR_ERR_INVALID_ARG;
  if (h->ws.sketch_kind && n != h->ws.dct_n) return SDR_ERR_INVALID_ARG;
  if (h->prec != SDR_PREC_F64) return SDR_ERR_NOT_IMPLEMENTED;
  if (kdim > 0 && !U) return SDR_ERR_INVALID_ARG;
  StreamGuard guard(h);
  if (kdim > 0 && !SAU && !csr_ok(h, A)) return SDR_ERR_INVALID_ARG;
  const WS& ws = h->ws;
  h->kh = kdim;
  if (kdim == 0) return SDR_OK;
  SDR_CK(cudaMemcpy2DAsync(ws.U[h->cu], ws.ldv * sizeof(double), U, n * sizeof(double), n * sizeof(double), kdim,
                           cudaMemcpyDeviceToDevice, h->st));
  {
    WS w2 = h->ws;
    w2.n = n;
    SDR_CK(launch_umax<double>(w2, (const double*)ws.U[h->cu], kdim, h->cu, h->st));
  }
  if (SU)
    SDR_CK(cudaMemcpyAsync(ws.SU[h->cu], SU, (size_t)ws.s * kdim * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  if (SAU)
    SDR_CK(cudaMemcpyAsync(ws.SAU[h->cu], SAU, (size_t)ws.s * kdim * sizeof(double), cudaMemcpyDeviceToDevice,
                           h->st));
  SDR_CK(cudaStreamSynchronize(h->st));
  if (!SU) {
    sdr_status s = recompute_su<double>(h, n);
    if (s != SDR_OK) return s;
  }
  if (!SAU) {
    const sdr_status s = recompute_sau<double>(h, A, n);
    if (s != SDR_OK) return s;
  }
  return verify_sau_rank(h);
}

}  // extern "C"
