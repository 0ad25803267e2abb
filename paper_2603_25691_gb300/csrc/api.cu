// C ABI and host orchestration of one unaligned kernel-mode PCG solve
// (Brust & Kolda, §4.4).  Declarations and argument conventions:
// include/cphifi.h.
//
// The solve runs in the eigenbasis of K: with K = U_K D_K U_K' (Eq. eigK) and
// X = U_K Xbar, the system of Eq. unaligned-infinite-1 becomes
//   Abar xbar = D_K U_K' Yhat1(U_K D_K Xbar) + (lambda D_K + rho) Xbar = bbar,
//   bbar = D_K U_K' B,
// where Yhat1(Xhat) is the gather-dot/scatter of Eqs. vl and yhat1.  The
// preconditioner of Eqs. precon/fx becomes the row-local r x r map
// ((Xbar U_V) .* D) U_V'.  Each iteration therefore reads the n x n matrix
// U_K twice (instead of K twice and U_K twice) and the operator built from a
// rounded U_K stays symmetric positive definite because U_K appears on both
// sides.  W = U_K Wbar at the end.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <tuple>
#include <string>
#include <utility>
#include <vector>

#include "cphifi.h"
#include "launch.h"

using namespace cphifi;

struct Request;
static void requests_clear(cphifi_ctx* ctx);

struct cphifi_ctx {
  int device = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  cudaStream_t user_stream = nullptr;
  bool has_user_stream = false;
  size_t budget = 0;
  size_t in_use = 0;
  std::string last_error;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  DevScalars* h_scalars = nullptr;  // pinned
  // Device blocks released by destroyed problems, by size: a new problem of a
  // similar shape reuses them instead of paying cudaMalloc/cudaFree (and the
  // device synchronisation cudaFree implies) on every solve.
  std::multimap<size_t, void*> pool;
  size_t pool_bytes = 0;
  // Pinned host slots (one per problem: its scalars and the tensor-core error
  // word) carved from page-locked slabs, and a free list of CUDA events, so
  // that creating a problem pins no memory and creates no event.
  std::vector<void*> pinned_slabs;
  std::vector<char*> pinned_free;
  std::vector<cudaEvent_t> events_free;
  // Temporaries of asynchronous problem creations, returned to the pool once
  // the event recorded after their last use has completed.
  std::vector<std::pair<cudaEvent_t, std::vector<std::pair<void*, size_t>>>> deferred;
  size_t deferred_bytes = 0;
  cudaEvent_t phase[4] = {nullptr, nullptr, nullptr, nullptr};  // solve phase marks
  // Second stream of the synchronous problem creation: Gram and eig(V) (one
  // block) overlap the observation passes on the main stream.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // Host-to-device stream of the chunked observation upload (§ zhat_and_rhs).
  cudaStream_t copy = nullptr;
  // Launch shapes per problem-size bucket (floor(log2 n), floor(log2 q), r),
  // set by cphifi_ctx_set_tuning (the autotuner); absent buckets use the
  // built-in heuristics.
  std::map<std::tuple<int, int, int>, cphifi_tuning> tuning;
  // Submitted requests (cphifi_submit): admitted FIFO while a slot (stream)
  // and the HBM budget allow, advanced by cphifi_poll / cphifi_wait.
  uint64_t next_ticket = 1;
  int max_active = 16;
  std::vector<cudaStream_t> slot_stream;
  std::vector<bool> slot_busy;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<uint64_t, Request*> requests;
  std::vector<uint64_t> done_unreported;  // completed, not yet listed by poll
  // Streams of the batch call's problem creations (created on first use) and
  // the events timing its persistent launch.
  std::vector<cudaStream_t> batch_streams;
  cudaEvent_t batch_ev[2] = {nullptr, nullptr};
  // bound of the persistent launch's idle wait: no tile finished anywhere
  long long batch_wait_ns = 4000000000ll;
};

struct cphifi_kernel {
  cphifi_ctx* ctx = nullptr;
  int n = 0;
  double* UK64 = nullptr;  // n x n column-major
  float* UK32 = nullptr;   // fl32(U_K): the FP32 operator's U_K and the hi part
  float* UKlo = nullptr;   // fl32(U_K - UK32): U_K = UK32 + UKlo to 2^-48 (double-float)
  // Tensor-core operand copies (leading dimension ldt = n rounded up to 8):
  // A1 = row-major U_K (A of U_K X), A2 = row-major U_K' (A of U_K' X).
  bool tc = false;
  int64_t ldt = 0;
  float *A1f = nullptr, *A2f = nullptr;
  __nv_bfloat16 *A1b = nullptr, *A2b = nullptr;
  float *A1h = nullptr, *A1l = nullptr, *A2h = nullptr, *A2l = nullptr;  // 3-term TF32 split
  CUtensorMap mA1f, mA2f, mA1b, mA2b, mA1h, mA1l, mA2h, mA2l;
  // BF16 slices of U_K and U_K' for the FP64-accurate tensor-core products
  // (oz_gemm.cu) and their row exponents (n for U_K, then n for U_K').
  bool oz = false;
  __nv_bfloat16 *oz1 = nullptr, *oz2 = nullptr;
  int* oze = nullptr;
  CUtensorMap mOz1, mOz2;
  double* dK = nullptr;    // n
  size_t bytes = 0;
  // design points (kernels created from points): K's entries are generated
  // from them in the products with K
  double* pts = nullptr;   // n x dim, row-major
  int dim = 0, kind = 0;
  double bandwidth = 0.0;
};

struct cphifi_problem {
  cphifi_ctx* ctx = nullptr;
  const cphifi_kernel* kern = nullptr;
  int n = 0, r = 0, d_other = 0;
  int64_t q = 0;
  double gamma = 0.0;
  std::vector<int64_t> sizes;
  std::vector<std::pair<void*, size_t>> allocs;
  size_t bytes = 0;
  // observation data (sorted by kernel index)
  int32_t* perm = nullptr;
  int64_t* row_ptr = nullptr;
  double* z64 = nullptr;  // Zhat in FP64 (the FP64 operator)
  // Zhat as an FP32 pair (mixed and double-float modes): one array of tiles
  // [hi block | lo block] (tile stride 64 r); zhi points at it, zlo = zhi + 32 r.
  float* zhi = nullptr;
  float* zlo = nullptr;
  int32_t *pseg = nullptr, *pbeg = nullptr, *pend = nullptr, *seg_first = nullptr,
          *seg_count = nullptr, *warp_first = nullptr;
  unsigned* seg_ticket = nullptr;
  unsigned* wctr = nullptr;  // dynamic work counters of the observation passes (2, zero)
  int npieces = 0;
  int nwarps = 1;     // warps of the gather-dot/scatter, L observations each
  int64_t obs_per_warp = 1;
  void* gds_partial = nullptr;  // npieces x 64 doubles
  // factors and their Gram
  std::vector<double*> factors;
  std::vector<float*> fhl;  // factors as row-major interleaved double-float pairs
  double** factors_dev = nullptr;
  float** fhl_dev = nullptr;
  int64_t* sizes_dev = nullptr;
  double *V = nullptr, *dV = nullptr, *UV = nullptr;
  float* UV32 = nullptr;
  int* info = nullptr;
  double* Bm = nullptr;  // sparse MTTKRP B (n x r, original basis)
  // solve workspace (n x r each)
  double *x = nullptr, *res = nullptr, *z = nullptr, *p = nullptr, *y = nullptr,
         *bbar = nullptr, *xh64 = nullptr, *y164 = nullptr, *tmp64 = nullptr,
         *tmp64b = nullptr, *D64 = nullptr;
  double* tres = nullptr;  // true residual of the mixed modes' periodic check
  float *pop32 = nullptr, *xh32 = nullptr, *y132 = nullptr, *D32 = nullptr;
  float *Bhi = nullptr, *Blo = nullptr;  // double-float product operand
  // Low-precision product operands pop (D_K P̄) and y1 (Ŷ1) use leading
  // dimension ldt (= the kernel's tensor-core ldt, else n); BF16 copies and
  // TMA maps for the tensor-core modes.
  int64_t ldt = 0;
  __nv_bfloat16 *pop16 = nullptr, *y116 = nullptr;
  float *poph = nullptr, *popl = nullptr, *y1h = nullptr, *y1l = nullptr;  // 3-term TF32 split
  CUtensorMap mBpf, mBpb, mByf, mByb, mBph, mBpl, mByh, mByl;
  // B slices of the FP64-accurate tensor-core products (when the kernel has
  // U_K slices) and their column exponents
  __nv_bfloat16* ozb = nullptr;
  int* ozce = nullptr;
  CUtensorMap mOzb;
  int nsplittc = 1;
  int* tc_err = nullptr;
  // Stream, pinned scalar copy and phase events of this problem's solves (the
  // context's stream for the synchronous calls, a pool stream for submitted
  // requests).
  cudaStream_t st = nullptr;
  DevScalars* hs = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  void* cpart = nullptr;  // max(nsplit64, nsplit32, nsplitdf) x n x r doubles
  int nsplit64 = 1, nsplit32 = 1, nsplitdf = 1;  // splits of the k range per product kind
  RedScratch red{};
  DevScalars* s = nullptr;    // the solve's scalars
  DevScalars* s2 = nullptr;   // scalars of the step-by-step calls
  int* err = nullptr;
  int64_t create_launches = 0;
  // alternating fit (CPHIFI_KEEP_OBS): observation lists in the sorted order,
  // per-finite-mode sort (built on first use), A_k = K W, and whether the
  // factors changed since Zhat / B / V were built.
  bool keep_obs = false;
  int32_t* kidx_s = nullptr;
  int32_t* oidx_s = nullptr;
  double* vals_s = nullptr;
  std::vector<int32_t*> perm_m;
  std::vector<int64_t*> rowp_m;
  double* Ak = nullptr;
  double* fit2 = nullptr;  // 2 doubles
  int* nfail = nullptr;
  bool stale = false;
  // Per-index Gram blocks C_i (gram.cu), n x r x r each, built on first use
  // and kept until the factors change: FP32 (the mixed operator) and
  // FP64-accurate (the FP64 operators and checks); the piece decomposition of
  // their build (L_g observations per piece) and its partial blocks.
  float* C32 = nullptr;
  double* C64 = nullptr;
  bool c32_ok = false, c64_ok = false;
  int32_t *gseg = nullptr, *gbeg = nullptr, *gend = nullptr, *gfirst = nullptr,
          *gcount = nullptr;
  unsigned* gticket = nullptr;
  double* gpart = nullptr;
  int gnp = 0;
};

// ------------------------------------------------------------ helpers -----
namespace {

int fail(cphifi_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

#define CK(...)                                                                          \
  do {                                                                                   \
    cudaError_t e_ = (__VA_ARGS__);                                                      \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, CPHIFI_E_DEVICE, std::string(#__VA_ARGS__ " failed: ") +         \
                                            cudaGetErrorString(e_));                     \
  } while (0)

struct Enter {
  // Orders the call after the caller's stream and makes the context's device
  // current for the duration of the call.
  cphifi_ctx* ctx;
  int prev = -1;
  explicit Enter(cphifi_ctx* c) : ctx(c) {
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    if (ctx->has_user_stream) {
      cudaEventRecord(ctx->ev_in, ctx->user_stream);
      cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0);
    }
  }
  ~Enter() {
    if (ctx->has_user_stream) {
      cudaEventRecord(ctx->ev_out, ctx->stream);
      cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0);
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  }
};

size_t pool_round(size_t bytes) {
  if (bytes <= 4096) return (bytes + 255) & ~(size_t)255;
  size_t g = 1;
  while (g * 2 <= bytes) g *= 2;
  const size_t step = std::max<size_t>(256, g / 8);
  return (bytes + step - 1) / step * step;
}

void pool_trim(cphifi_ctx* ctx) {
  for (auto& kv : ctx->pool) cudaFree(kv.second);
  ctx->pool.clear();
  ctx->pool_bytes = 0;
}

// A block of at least `bytes` (rounded to a size class) from the pool, or a
// new one; *got is the block's size.
cudaError_t pool_alloc(cphifi_ctx* ctx, size_t bytes, void** out, size_t* got) {
  const size_t want = pool_round(bytes ? bytes : 1);
  auto it = ctx->pool.lower_bound(want);
  if (it != ctx->pool.end() && it->first <= want + want / 4) {
    *out = it->second;
    *got = it->first;
    ctx->pool_bytes -= it->first;
    ctx->pool.erase(it);
    return cudaSuccess;
  }
  if (ctx->budget && ctx->in_use + ctx->pool_bytes + want > ctx->budget) pool_trim(ctx);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pool_trim(ctx);
    e = cudaMalloc(&p, want);
  }
  if (e != cudaSuccess) return e;
  *out = p;
  *got = want;
  return cudaSuccess;
}

void pool_release(cphifi_ctx* ctx, void* p, size_t bytes) {
  ctx->pool.emplace(bytes, p);
  ctx->pool_bytes += bytes;
}

template <typename T>
cudaError_t dalloc(cphifi_problem* P, T** out, size_t count) {
  *out = nullptr;
  if (count == 0) count = 1;
  void* p = nullptr;
  size_t got = 0;
  cudaError_t e = pool_alloc(P->ctx, count * sizeof(T), &p, &got);
  if (e != cudaSuccess) return e;
  P->allocs.push_back({p, got});
  P->bytes += got;
  P->ctx->in_use += got;
  *out = (T*)p;
  return cudaSuccess;
}

constexpr size_t kPinnedSlot = 256;
constexpr int kPinnedPerSlab = 64;
static_assert(sizeof(DevScalars) + 16 <= kPinnedSlot, "pinned slot too small");

cudaError_t pinned_get(cphifi_ctx* ctx, void** out) {
  if (ctx->pinned_free.empty()) {
    void* slab = nullptr;
    cudaError_t e = cudaMallocHost(&slab, kPinnedSlot * kPinnedPerSlab);
    if (e != cudaSuccess) return e;
    ctx->pinned_slabs.push_back(slab);
    for (int k = kPinnedPerSlab - 1; k >= 0; --k)
      ctx->pinned_free.push_back((char*)slab + k * kPinnedSlot);
  }
  *out = ctx->pinned_free.back();
  ctx->pinned_free.pop_back();
  return cudaSuccess;
}

cudaError_t event_get(cphifi_ctx* ctx, cudaEvent_t* out) {
  if (!ctx->events_free.empty()) {
    *out = ctx->events_free.back();
    ctx->events_free.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(out);
}

// Returns deferred temporaries whose last use has completed (all of them,
// after a wait, when `wait` is set).
void deferred_collect(cphifi_ctx* ctx, bool wait) {
  auto& d = ctx->deferred;
  size_t k = 0;
  for (size_t i = 0; i < d.size(); ++i) {
    // after a wait the entry is released whatever the query says
    const bool done = wait ? (cudaEventSynchronize(d[i].first), true)
                           : cudaEventQuery(d[i].first) == cudaSuccess;
    if (done) {
      for (auto& t : d[i].second) {
        pool_release(ctx, t.first, t.second);
        ctx->deferred_bytes -= std::min(ctx->deferred_bytes, t.second);
      }
      ctx->events_free.push_back(d[i].first);
    } else {
      if (k != i) d[k] = std::move(d[i]);  // (a self-move would empty the list)
      ++k;
    }
  }
  d.resize(k);
  if (d.empty()) ctx->deferred_bytes = 0;
}

const char* input_error_text(int herr) {
  if (herr & 1) return "observation index out of range";
  if (herr & 2) return "non-finite observation value or factor entry";
  if (herr & 4) return "CPHIFI_OBS_SORTED set but kidx is not sorted";
  return "invalid observation data";
}

void free_problem(cphifi_problem* P) {
  if (P->hs) P->ctx->pinned_free.push_back((char*)P->hs);
  P->hs = nullptr;
  for (auto& e : P->ev)
    if (e) { P->ctx->events_free.push_back(e); e = nullptr; }
  for (auto& a : P->allocs) pool_release(P->ctx, a.first, a.second);
  P->ctx->in_use -= std::min(P->ctx->in_use, P->bytes);
  P->allocs.clear();
  P->bytes = 0;
}

// Kernel count of a launcher call as written in problem_create (the scan
// launches three kernels, each radix pass three plus the scan's three).
bool is_launch(const char* call) {
  return strncmp(call, "launch_", 7) == 0 || strncmp(call, "radix_sort_pairs", 16) == 0 ||
         strncmp(call, "exclusive_scan_i32", 18) == 0;
}
int64_t launch_weight(const char* call) {
  if (strncmp(call, "exclusive_scan_i32", 18) == 0) return 3;
  if (strncmp(call, "radix_sort_pairs", 16) == 0) return 10;
  return 1;
}

int bits_for(int n) {
  int b = 1;
  while (b < 31 && (1LL << b) < n) ++b;
  return b;
}

// Copies `bytes` from a caller buffer (host or device) into device memory.
cudaError_t upload(void* dst, const void* src, size_t bytes, int mem, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes,
                         mem == CPHIFI_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyHostToDevice,
                         st);
}

cudaError_t download(void* dst, const void* src, size_t bytes, int mem, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes,
                         mem == CPHIFI_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyDeviceToHost,
                         st);
}

// Launch timing: pairs of events around selected launches.
struct Timer {
  cudaStream_t st;
  bool on;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gds, gemm, gds64, gemm64;
  std::vector<cudaEvent_t> pool;
  Timer(cudaStream_t s, bool enabled) : st(s), on(enabled) {}
  ~Timer() {
    for (auto e : pool) cudaEventDestroy(e);
  }
  Timer(const Timer&) = delete;
  Timer& operator=(const Timer&) = delete;
  cudaEvent_t ev() {
    cudaEvent_t e;
    cudaEventCreate(&e);
    pool.push_back(e);
    return e;
  }
  cudaEvent_t begin() {
    if (!on) return nullptr;
    cudaEvent_t e = ev();
    cudaEventRecord(e, st);
    return e;
  }
  void end(cudaEvent_t b, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v) {
    if (!on) return;
    cudaEvent_t e = ev();
    cudaEventRecord(e, st);
    v.push_back({b, e});
  }
  static double total(const std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v) {
    double t = 0;
    for (auto& pr : v) {
      float ms = 0;
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      t += ms;
    }
    return t;
  }
};

}  // namespace

// ----------------------------------------------------------- context ------
extern "C" const char* cphifi_status_string(int status) {
  switch (status) {
    case CPHIFI_OK: return "ok";
    case CPHIFI_E_INVALID_ARG: return "invalid argument";
    case CPHIFI_E_OOM: return "device allocation failed";
    case CPHIFI_E_ADMISSION: return "footprint exceeds the HBM budget";
    case CPHIFI_E_NOT_CONVERGED: return "not converged within max_iter";
    case CPHIFI_E_BREAKDOWN: return "PCG breakdown (p'Ap <= 0 or non-finite scalar)";
    case CPHIFI_E_DEVICE: return "CUDA error";
    case CPHIFI_E_TIMEOUT: return "timed out";
    case CPHIFI_E_UNSUPPORTED: return "unsupported in this build";
    default: return "unknown status";
  }
}

extern "C" int cphifi_ctx_create(cphifi_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return CPHIFI_E_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = new cphifi_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  bool ok = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) == cudaSuccess &&
            cudaMallocHost(&ctx->h_scalars, sizeof(DevScalars)) == cudaSuccess;
  for (int k = 0; ok && k < 4; ++k) ok = cudaEventCreate(&ctx->phase[k]) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) == cudaSuccess;
  cudaSetDevice(prev);
  if (!ok) {
    delete ctx;
    return CPHIFI_E_DEVICE;
  }
  *out = ctx;
  return CPHIFI_OK;
}

extern "C" int cphifi_ctx_destroy(cphifi_ctx* ctx) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  requests_clear(ctx);
  deferred_collect(ctx, true);
  pool_trim(ctx);
  for (auto e : ctx->phase)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  if (ctx->copy) {
    cudaStreamSynchronize(ctx->copy);
    cudaStreamDestroy(ctx->copy);
  }
  for (auto bs : ctx->batch_streams) {
    cudaStreamSynchronize(bs);
    cudaStreamDestroy(bs);
  }
  for (auto e : ctx->batch_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->h_scalars) cudaFreeHost(ctx->h_scalars);
  for (auto e : ctx->events_free) cudaEventDestroy(e);
  for (auto p : ctx->pinned_slabs) cudaFreeHost(p);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaSetDevice(prev);
  delete ctx;
  return CPHIFI_OK;
}

extern "C" int cphifi_ctx_set_stream(cphifi_ctx* ctx, void* stream) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  ctx->user_stream = (cudaStream_t)stream;
  ctx->has_user_stream = true;
  return CPHIFI_OK;
}

extern "C" size_t cphifi_ctx_bytes_in_use(const cphifi_ctx* ctx) { return ctx ? ctx->in_use : 0; }

extern "C" const char* cphifi_last_error(const cphifi_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "null context";
}

// ------------------------------------------------------------ kernel ------
extern "C" int cphifi_kernel_create(cphifi_ctx* ctx, int64_t n, const double* K,
                                    const double* UK, const double* DK, int mem,
                                    cphifi_kernel** out) {
  if (!ctx || !out) return CPHIFI_E_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || n > (1 << 20)) return fail(ctx, CPHIFI_E_INVALID_ARG, "n out of range");
  const bool device_eig = !UK && !DK;
  if (device_eig && !K)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "either K or its eigendecomposition (UK, DK) is needed");
  if (!device_eig && (!UK || !DK))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "UK and DK are passed together");
  if (device_eig && n > kSymEigMaxN)
    return fail(ctx, CPHIFI_E_UNSUPPORTED,
                "n too large for the device eigensolver (n <= " + std::to_string(kSymEigMaxN) +
                    "): pass UK and DK");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  const size_t nn = (size_t)n * n;
  const size_t bytes = nn * (sizeof(double) + 2 * sizeof(float)) + n * sizeof(double);
  if (ctx->budget && ctx->in_use + bytes > ctx->budget)
    return fail(ctx, CPHIFI_E_ADMISSION, "kernel matrix exceeds the HBM budget");
  Enter guard(ctx);
  cphifi_kernel* kern = new cphifi_kernel();
  kern->ctx = ctx;
  kern->n = (int)n;
  int* err = nullptr;
  auto cleanup = [&](int code, const std::string& m) {
    if (kern->UK64) cudaFree(kern->UK64);
    if (kern->UK32) cudaFree(kern->UK32);
    if (kern->UKlo) cudaFree(kern->UKlo);
    if (kern->dK) cudaFree(kern->dK);
    for (void* a : {(void*)kern->A1f, (void*)kern->A2f, (void*)kern->A1b, (void*)kern->A2b,
                    (void*)kern->A1h, (void*)kern->A1l, (void*)kern->A2h, (void*)kern->A2l,
                    (void*)kern->oz1, (void*)kern->oz2, (void*)kern->oze})
      if (a) cudaFree(a);
    if (err) cudaFree(err);
    delete kern;
    return fail(ctx, code, m);
  };
  if (cudaMalloc(&kern->UK64, nn * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&kern->UK32, nn * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&kern->UKlo, nn * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&kern->dK, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess)
    return cleanup(CPHIFI_E_OOM, "cudaMalloc failed for the kernel matrix");
  cudaStream_t st = ctx->stream;
  int herr = 0;
  if (device_eig) {  // K = U_K diag(D_K) U_K' on the device (Eq. eigK), FP64
    if (upload(kern->UK64, K, nn * sizeof(double), mem, st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
        launch_validate_dense(kern->UK64, (int64_t)nn, err, st) != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return cleanup(CPHIFI_E_DEVICE, "uploading K failed");
    if (herr) return cleanup(CPHIFI_E_INVALID_ARG, "non-finite entry in K");
    std::string why;
    const int rc = sym_eig_jacobi(kern->UK64, (int)n, kern->dK, st, &why);
    if (rc != CPHIFI_OK) return cleanup(rc, why);
  }
  if ((!device_eig && (upload(kern->UK64, UK, nn * sizeof(double), mem, st) != cudaSuccess ||
                       upload(kern->dK, DK, n * sizeof(double), mem, st) != cudaSuccess)) ||
      cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
      launch_validate_dense(kern->UK64, (int64_t)nn, err, st) != cudaSuccess ||
      launch_validate_dense(kern->dK, n, err, st) != cudaSuccess ||
      launch_split_df(kern->UK64, nullptr, (int64_t)nn, (int64_t)nn, kern->UK32, kern->UKlo, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cleanup(CPHIFI_E_DEVICE, "uploading the kernel eigendecomposition failed");
  if (herr) return cleanup(CPHIFI_E_INVALID_ARG, "non-finite entry in UK or DK");
  size_t tc_bytes = 0;
  if (tc_available((int)n)) {
    const int64_t ldt = (n + 7) / 8 * 8;
    const size_t cnt = (size_t)n * ldt;
    tc_bytes = cnt * (6 * sizeof(float) + 2 * sizeof(__nv_bfloat16));
    if (ctx->budget && ctx->in_use + bytes + tc_bytes > ctx->budget) {
      tc_bytes = 0;  // no room: the tensor-core modes stay unavailable
    } else if (cudaMalloc(&kern->A1f, cnt * sizeof(float)) == cudaSuccess &&
               cudaMalloc(&kern->A2f, cnt * sizeof(float)) == cudaSuccess &&
               cudaMalloc(&kern->A1b, cnt * sizeof(__nv_bfloat16)) == cudaSuccess &&
               cudaMalloc(&kern->A2b, cnt * sizeof(__nv_bfloat16)) == cudaSuccess &&
               cudaMalloc(&kern->A1h, cnt * sizeof(float)) == cudaSuccess &&
               cudaMalloc(&kern->A1l, cnt * sizeof(float)) == cudaSuccess &&
               cudaMalloc(&kern->A2h, cnt * sizeof(float)) == cudaSuccess &&
               cudaMalloc(&kern->A2l, cnt * sizeof(float)) == cudaSuccess &&
               launch_uk_copy<float>(kern->UK64, (int)n, ldt, true, kern->A1f, st) == cudaSuccess &&
               launch_uk_copy<float>(kern->UK64, (int)n, ldt, false, kern->A2f, st) == cudaSuccess &&
               launch_uk_copy<__nv_bfloat16>(kern->UK64, (int)n, ldt, true, kern->A1b, st) == cudaSuccess &&
               launch_uk_copy<__nv_bfloat16>(kern->UK64, (int)n, ldt, false, kern->A2b, st) == cudaSuccess &&
               tc_make_map(&kern->mA1f, kern->A1f, false, n, n, ldt * 4, 128) == cudaSuccess &&
               tc_make_map(&kern->mA2f, kern->A2f, false, n, n, ldt * 4, 128) == cudaSuccess &&
               tc_make_map(&kern->mA1b, kern->A1b, true, n, n, ldt * 2, 128) == cudaSuccess &&
               tc_make_map(&kern->mA2b, kern->A2b, true, n, n, ldt * 2, 128) == cudaSuccess &&
               launch_tf32_split(kern->A1f, kern->A1h, kern->A1l, (int64_t)cnt, st) == cudaSuccess &&
               launch_tf32_split(kern->A2f, kern->A2h, kern->A2l, (int64_t)cnt, st) == cudaSuccess &&
               tc_make_map(&kern->mA1h, kern->A1h, false, n, n, ldt * 4, 128) == cudaSuccess &&
               tc_make_map(&kern->mA1l, kern->A1l, false, n, n, ldt * 4, 128) == cudaSuccess &&
               tc_make_map(&kern->mA2h, kern->A2h, false, n, n, ldt * 4, 128) == cudaSuccess &&
               tc_make_map(&kern->mA2l, kern->A2l, false, n, n, ldt * 4, 128) == cudaSuccess &&
               cudaStreamSynchronize(st) == cudaSuccess) {
      kern->tc = true;
      kern->ldt = ldt;
    } else {
      cudaGetLastError();
      return cleanup(CPHIFI_E_DEVICE, "building the tensor-core copies of U_K failed");
    }
    // slices for the FP64-accurate products, when the budget has room (else
    // those products stay on the double-float SIMT kernel)
    const size_t oz_bytes = oz_uk_bytes((int)n, ldt);
    if (!ctx->budget || ctx->in_use + bytes + tc_bytes + oz_bytes <= ctx->budget) {
      const size_t sb = (size_t)oz_mpad((int)n) * ldt * 7 * sizeof(__nv_bfloat16);
      const bool got = cudaMalloc(&kern->oz1, sb) == cudaSuccess &&
                       cudaMalloc(&kern->oz2, sb) == cudaSuccess &&
                       cudaMalloc(&kern->oze, 2 * (size_t)n * sizeof(int)) == cudaSuccess;
      if (!got) {  // no room on the device: the double-float products serve instead
        cudaGetLastError();
        for (void** a : {(void**)&kern->oz1, (void**)&kern->oz2, (void**)&kern->oze})
          if (*a) {
            cudaFree(*a);
            *a = nullptr;
          }
      } else if (launch_oz_uk(kern->UK64, (int)n, ldt, kern->oz1, kern->oz2, kern->oze, st) ==
                     cudaSuccess &&
                 oz_make_maps(kern->oz1, kern->oz2, (int)n, ldt, &kern->mOz1, &kern->mOz2) ==
                     cudaSuccess &&
                 cudaStreamSynchronize(st) == cudaSuccess) {
        kern->oz = true;
        tc_bytes += oz_bytes;
      } else {
        cudaGetLastError();
        return cleanup(CPHIFI_E_DEVICE, "building the tensor-core slices of U_K failed");
      }
    }
  }
  cudaFree(err);
  kern->bytes = bytes + (kern->tc ? tc_bytes : 0);
  ctx->in_use += kern->bytes;
  *out = kern;
  return CPHIFI_OK;
}

static bool kernel_in_use(const cphifi_ctx* ctx, const cphifi_kernel* kern);

extern "C" int cphifi_kernel_destroy(cphifi_kernel* kern) {
  if (!kern) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = kern->ctx;
  if (kernel_in_use(ctx, kern))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "kernel still used by submitted requests");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(kern->UK64);
  cudaFree(kern->UK32);
  cudaFree(kern->UKlo);
  cudaFree(kern->dK);
  for (void* a : {(void*)kern->A1f, (void*)kern->A2f, (void*)kern->A1b, (void*)kern->A2b,
                  (void*)kern->A1h, (void*)kern->A1l, (void*)kern->A2h, (void*)kern->A2l,
                  (void*)kern->oz1, (void*)kern->oz2, (void*)kern->oze})
    if (a) cudaFree(a);
  if (kern->pts) cudaFree(kern->pts);
  ctx->in_use -= std::min(ctx->in_use, kern->bytes);
  cudaSetDevice(prev);
  delete kern;
  return CPHIFI_OK;
}

extern "C" int cphifi_kernel_create_points(cphifi_ctx* ctx, int64_t n, int32_t dim,
                                           const double* x, int32_t kind, double bandwidth,
                                           int mem, cphifi_kernel** out) {
  if (!ctx || !out || !x) return CPHIFI_E_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || n > kSymEigMaxN)
    return fail(ctx, n < 1 ? CPHIFI_E_INVALID_ARG : CPHIFI_E_UNSUPPORTED,
                "n must be in [1, " + std::to_string(kSymEigMaxN) + "] (device eigensolver)");
  if (dim < 1 || dim > 64) return fail(ctx, CPHIFI_E_INVALID_ARG, "dim must be in [1, 64]");
  if (kind != CPHIFI_KERNEL_GAUSSIAN && kind != CPHIFI_KERNEL_MATERN32)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "unknown kernel kind");
  if (!(bandwidth > 0.0) || !std::isfinite(bandwidth))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "bandwidth must be finite and > 0");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  const size_t npts = (size_t)n * dim;
  if (ctx->budget && ctx->in_use + (size_t)n * n * sizeof(double) + npts * sizeof(double) >
                         ctx->budget)
    return fail(ctx, CPHIFI_E_ADMISSION, "kernel matrix exceeds the HBM budget");
  Enter guard(ctx);
  cudaStream_t st = ctx->stream;
  double* pts = nullptr;
  double* K = nullptr;
  int* err = nullptr;
  int herr = 0;
  auto bail = [&](int code, const std::string& m) {
    cudaStreamSynchronize(st);
    if (pts) cudaFree(pts);
    if (K) cudaFree(K);
    if (err) cudaFree(err);
    return fail(ctx, code, m);
  };
  if (cudaMalloc(&pts, npts * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&K, (size_t)n * n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess)
    return bail(CPHIFI_E_OOM, "cudaMalloc failed for the points or K");
  if (upload(pts, x, npts * sizeof(double), mem, st) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
      launch_validate_dense(pts, (int64_t)npts, err, st) != cudaSuccess ||
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return bail(CPHIFI_E_DEVICE, "uploading the points failed");
  if (herr) return bail(CPHIFI_E_INVALID_ARG, "non-finite point coordinate");
  if (launch_kpoints_build(pts, (int)n, dim, kind, bandwidth, K, st) != cudaSuccess)
    return bail(CPHIFI_E_DEVICE, "building K from the points failed");
  cphifi_kernel* kern = nullptr;
  const int rc = cphifi_kernel_create(ctx, n, K, nullptr, nullptr, CPHIFI_MEM_DEVICE, &kern);
  cudaFree(K);
  K = nullptr;
  cudaFree(err);
  err = nullptr;
  if (rc != CPHIFI_OK) {
    cudaFree(pts);
    return rc;
  }
  kern->pts = pts;
  kern->dim = dim;
  kern->kind = kind;
  kern->bandwidth = bandwidth;
  kern->bytes += npts * sizeof(double);
  ctx->in_use += npts * sizeof(double);
  *out = kern;
  return CPHIFI_OK;
}

extern "C" int cphifi_kernel_apply(const cphifi_kernel* kern, int32_t precision, int32_t r,
                                   const double* X, double* Y, int mem) {
  if (!kern || !X || !Y) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = kern->ctx;
  if (r < 1 || r > kMaxRank) return fail(ctx, CPHIFI_E_INVALID_ARG, "r must be in [1, 64]");
  if (precision != CPHIFI_FP64 && precision != CPHIFI_MIXED_FP32)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "precision must be FP64 or MIXED_FP32");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  Enter guard(ctx);
  cudaStream_t st = ctx->stream;
  const int n = kern->n;
  const size_t nr = (size_t)n * r;
  double *Xd = nullptr, *Yd = nullptr, *T = nullptr;
  auto done = [&](int code, const char* m) {
    cudaStreamSynchronize(st);
    if (mem != CPHIFI_MEM_DEVICE) {
      if (Xd) cudaFree(Xd);
      if (Yd) cudaFree(Yd);
    }
    if (T) cudaFree(T);
    return code == CPHIFI_OK ? code : fail(ctx, code, m);
  };
  if (mem == CPHIFI_MEM_DEVICE) {
    Xd = const_cast<double*>(X);
    Yd = Y;
  } else if (cudaMalloc(&Xd, nr * sizeof(double)) != cudaSuccess ||
             cudaMalloc(&Yd, nr * sizeof(double)) != cudaSuccess ||
             cudaMemcpyAsync(Xd, X, nr * sizeof(double), cudaMemcpyHostToDevice, st) !=
                 cudaSuccess) {
    return done(CPHIFI_E_OOM, "staging X and Y failed");
  }
  cudaError_t e;
  if (kern->pts) {
    const int ns = kpoints_pick_split(n, ctx->num_sms);
    e = ns > 1 ? cudaMalloc(&T, (size_t)ns * nr * sizeof(double)) : cudaSuccess;
    if (e == cudaSuccess)
      e = launch_kpoints_apply(precision == CPHIFI_FP64, kern->pts, n, kern->dim, kern->kind,
                               kern->bandwidth, r, Xd, Yd, ns, T, st);
  } else {  // Y = U_K (D_K o (U_K' X)), FP64
    e = cudaMalloc(&T, nr * sizeof(double));
    if (e == cudaSuccess)
      e = launch_gemm_skinny<double, double>(kern->UK64, n, false, nullptr, Xd, n, T, n,
                                             (int64_t)nr, n, r, 1, nullptr, st);
    if (e == cudaSuccess)
      e = launch_gemm_skinny<double, double>(kern->UK64, n, true, kern->dK, T, n, Yd, n,
                                             (int64_t)nr, n, r, 1, nullptr, st);
  }
  if (e == cudaSuccess && mem != CPHIFI_MEM_DEVICE)
    e = cudaMemcpyAsync(Y, Yd, nr * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return done(CPHIFI_E_DEVICE, "kernel_apply failed");
  }
  return done(CPHIFI_OK, "");
}

extern "C" int cphifi_kernel_eig(const cphifi_kernel* kern, double* UK, double* DK, int mem) {
  if (!kern) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = kern->ctx;
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  Enter guard(ctx);
  const size_t n = (size_t)kern->n;
  if (UK) CK(download(UK, kern->UK64, n * n * sizeof(double), mem, ctx->stream));
  if (DK) CK(download(DK, kern->dK, n * sizeof(double), mem, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CPHIFI_OK;
}

// ----------------------------------------------------------- problem ------
// The chunked upload of host observations (problem_create_on): sorted lists
// of at least kPipelineMinQ observations, in kUploadChunks chunks.
constexpr int64_t kPipelineMinQ = int64_t(1) << 20;
constexpr int kUploadChunks = 8;

// Warps of the gather-dot/scatter decomposition: at most two resident 8-warp
// blocks per SM, and enough that no warp walks more than about 8 pieces
// (every kernel index, even an empty one, is a piece: with n > q most pieces
// are empty, and a warp takes its pieces one after another) while keeping at
// least 64 observations per warp when there are few indices.
static int64_t gds_warps(int num_sms, int64_t n, int64_t q, int warps_per_sm = 16) {
  const int64_t by_obs = (q + 63) / 64, by_pieces = (q + n + 7) / 8;
  return std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms * warps_per_sm,
                                                std::max(by_obs, std::min(by_pieces, q))));
}

static int floor_log2(int64_t v) {
  int b = 0;
  while (v > 1) {
    v >>= 1;
    ++b;
  }
  return b;
}

// Launch shapes of a problem: the gather-dot/scatter's warps and the k-range
// splits of the n x n products, from the context's tuning table when it has
// an entry for the problem's bucket, else from the heuristics.  Tuned splits
// are clamped to what each product kernel supports.
struct Shapes {
  int64_t W;
  int s64, s32, sdf, stc;
};
static Shapes problem_shapes(const cphifi_ctx* ctx, const cphifi_kernel* kern, int n, int64_t q,
                             int r) {
  cphifi_tuning t{};
  auto it = ctx->tuning.find(std::make_tuple(floor_log2(n), floor_log2(std::max<int64_t>(q, 1)), r));
  if (it != ctx->tuning.end()) t = it->second;
  const int sms = ctx->num_sms;
  auto pick = [](int tuned, int dflt, int cap) {
    return tuned > 0 ? std::max(1, std::min(tuned, cap)) : dflt;
  };
  Shapes sh;
  sh.W = gds_warps(sms, n, q, t.gds_warps_per_sm > 0 ? t.gds_warps_per_sm : 16);
  sh.s64 = pick(t.split64, gemm_pick_split<double, double>(n, sms), std::min(32, (n + 31) / 32));
  sh.s32 = pick(t.split32, gemm_pick_split<float, float>(n, sms), std::min(32, (n + 31) / 32));
  sh.sdf = kern->oz ? pick(t.split_wide, oz_pick_split(n, sms), std::min(64, (n + 255) / 256))
                    : pick(t.split_wide, gemm_df_pick_split(n, sms), std::min(32, (n + 15) / 16));
  sh.stc = kern->tc ? pick(t.split_tc, tc_pick_split(n, sms), std::min(64, (n + 31) / 32)) : 1;
  return sh;
}

static size_t problem_footprint(int64_t n, int64_t q, int r, int d_other,
                                const std::vector<int64_t>& sizes, bool lowp, int nsplit,
                                int64_t npieces_max) {
  size_t b = 0;
  const size_t nr = (size_t)n * r;
  b += (size_t)zhat_elems(q, r) * 2 * sizeof(float);  // Zhat hi + lo
  (void)lowp;
  b += (size_t)q * sizeof(int32_t);                    // perm
  b += (n + 1) * sizeof(int64_t) + 4 * n * sizeof(int32_t) + (n + 1) * sizeof(int32_t);
  b += (size_t)npieces_max * (3 * sizeof(int32_t) + 64 * sizeof(double));
  for (int m = 0; m < d_other; ++m) b += (size_t)sizes[m] * r * sizeof(double);
  b += 13 * nr * sizeof(double) + 4 * nr * sizeof(float);
  b += (size_t)nsplit * nr * sizeof(double);
  b += (size_t)kRedMaxBlocks * kRedSlots * sizeof(double);
  return b;
}

// Device bytes a problem holds (`need`) and the temporaries of its creation
// (`tmp`), for admission against the context's HBM budget.
static void problem_need(const cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                         const std::vector<int64_t>& sizes, int32_t r, int64_t q, uint32_t flags,
                         size_t* need, size_t* tmp) {
  const int n = kern->n;
  const bool tc = kern->tc;
  const Shapes sh = problem_shapes(ctx, kern, n, q, r);
  const int64_t npieces_max = (int64_t)n + sh.W + 1;
  const int nsplit = std::max(std::max(sh.s64, sh.s32), std::max(sh.sdf, sh.stc));
  const bool need64 = (flags & CPHIFI_NEED_FP64) || !(flags & CPHIFI_NEED_LOWP);
  const bool lowp = (flags & CPHIFI_NEED_LOWP) || !(flags & CPHIFI_NEED_FP64);
  *need = problem_footprint(n, q, r, d_other, sizes, lowp, nsplit, npieces_max) +
          (need64 ? (size_t)zhat_elems(q, r) * sizeof(double) : 0) +
          (tc ? oz_b_bytes(r, ((int64_t)n + 7) / 8 * 8) : 0);  // B slices
  *tmp = (size_t)q * (sizeof(int32_t) * (1 + d_other) + sizeof(double) * 3 + sizeof(uint32_t)) +
         radix_sort_tmp_bytes(q);  // index/value copies, sort keys, double-float values
  if (flags & CPHIFI_KEEP_OBS)  // sorted observation lists + A_k
    *need += (size_t)q * (sizeof(int32_t) * (1 + d_other) + sizeof(double)) +
             (size_t)n * r * sizeof(double);
}

// Zhat and the right-hand side MTTKRP B in one pass (zhat_mttkrp_kernel) over
// a second decomposition of the sorted observations into ranges of 256
// (8 tiles), which the warps draw in order: at any time they all write into a
// narrow window of the Zhat array, as the separate build does with its tile
// chunks.  The decomposition's arrays come from `alloc` (the caller's
// temporaries, free once the stream has passed this work).
// The Zhat pass's decomposition: W2 ranges of L2 observations, 256 each; more
// (and shorter) ranges when the kernel indices outnumber the observations,
// so that no warp walks long runs of empty pieces (as in gds_warps).
static void zhat_ranges(int num_sms, int64_t n, int64_t q, int64_t* W2, int64_t* L2) {
  *W2 = std::max<int64_t>(
      (q + 255) / 256, std::min<int64_t>(std::min<int64_t>((q + n + 7) / 8, q), (int64_t)num_sms * 16));
  *L2 = (q + *W2 - 1) / *W2;
}

// Chunks of a pipelined upload: chunk c covers the ranges [c W2 / K, (c+1) W2 /
// K), i.e. the observations [w0 L2, min(q, w1 L2)) -- pieces never cross a
// range boundary, so a chunk's ranges read only that chunk's observations.
static void zhat_chunk(int64_t W2, int64_t L2, int64_t q, int K, int c, int64_t* w0, int64_t* w1,
                       int64_t* o0, int64_t* o1) {
  *w0 = c * W2 / K;
  *w1 = (c + 1) * W2 / K;
  *o0 = std::min<int64_t>(q, *w0 * L2);
  *o1 = std::min<int64_t>(q, *w1 * L2);
}

// With `chunk_ready` (K events), the pass runs as K launches, launch c after
// event c (the upload of its chunk of other-mode indices and values).
template <typename Alloc>
static cudaError_t zhat_and_rhs(cphifi_problem* P, const int32_t* perm, const int32_t* oidx,
                                const double* vals, const int* gate, Alloc alloc,
                                cudaStream_t st,
                                const std::vector<cudaEvent_t>* chunk_ready = nullptr) {
  const int n = P->n;
  const int64_t q = P->q;
  if (q == 0) return cudaMemsetAsync(P->Bm, 0, (size_t)n * P->r * sizeof(double), st);
  int64_t W2 = 0, L2 = 0;
  zhat_ranges(P->ctx->num_sms, n, q, &W2, &L2);
  const int64_t np2 = (int64_t)n + W2 + 1;
  int32_t* cnt2 = (int32_t*)alloc((size_t)n * sizeof(int32_t));
  int32_t* first2 = (int32_t*)alloc((size_t)(n + 1) * sizeof(int32_t));
  int32_t* pseg2 = (int32_t*)alloc((size_t)np2 * sizeof(int32_t));
  int32_t* pbeg2 = (int32_t*)alloc((size_t)np2 * sizeof(int32_t));
  int32_t* pend2 = (int32_t*)alloc((size_t)np2 * sizeof(int32_t));
  int32_t* wfirst2 = (int32_t*)alloc((size_t)(W2 + 1) * sizeof(int32_t));
  unsigned* ticket2 = (unsigned*)alloc((size_t)n * sizeof(unsigned));
  double* partial2 = (double*)alloc((size_t)np2 * 64 * sizeof(double));
  void* stmp2 = alloc(exclusive_scan_tmp_bytes(n));
  if (!cnt2 || !first2 || !pseg2 || !pbeg2 || !pend2 || !wfirst2 || !ticket2 || !partial2 ||
      !stmp2)
    return cudaErrorMemoryAllocation;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ticket2, 0, (size_t)n * sizeof(unsigned), st)) != cudaSuccess ||
      (e = launch_piece_counts(P->row_ptr, n, L2, cnt2, gate, st)) != cudaSuccess ||
      (e = exclusive_scan_i32(cnt2, first2, n, stmp2, exclusive_scan_tmp_bytes(n), st)) !=
          cudaSuccess ||
      (e = launch_piece_fill(P->row_ptr, n, L2, first2, cnt2, pseg2, pbeg2, pend2, gate, st)) !=
          cudaSuccess ||
      (e = launch_warp_first(pbeg2, (int)np2, first2 + n, L2, (int)W2, wfirst2, gate, st)) !=
          cudaSuccess)
    return e;
  const PieceList pl2{pseg2, pbeg2, pend2, first2, cnt2, ticket2, wfirst2, (int)np2, (int)W2,
                      P->wctr};
  if (!chunk_ready)
    return launch_zhat_mttkrp_fused(pl2, q, perm, oidx, P->d_other, P->fhl_dev, P->sizes_dev,
                                    P->r, vals, P->zhi, P->z64, partial2, P->Bm, n, P->err, gate,
                                    P->ctx->num_sms, st);
  const int K = (int)chunk_ready->size();
  for (int c = 0; c < K; ++c) {
    int64_t w0, w1, o0, o1;
    zhat_chunk(W2, L2, q, K, c, &w0, &w1, &o0, &o1);
    if ((e = cudaStreamWaitEvent(st, (*chunk_ready)[c], 0)) != cudaSuccess ||
        (e = launch_zhat_mttkrp_fused(pl2, q, perm, oidx, P->d_other, P->fhl_dev, P->sizes_dev,
                                      P->r, vals, P->zhi, P->z64, partial2, P->Bm, n, P->err,
                                      gate, P->ctx->num_sms, st, (int)w0, (int)w1)) !=
            cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

// Problem creation on stream `st` (the context's stream for the public call, a
// pool stream for submitted requests).
// The device work is queued without host waits: the kernels after the input
// validation check the problem's error word before touching memory, the piece
// arrays take their upper bound (the exact count stays on the device).  A
// synchronous creation then waits once, reads the error word and returns the
// temporaries to the pool.  With `async` set (submitted requests) nothing
// waits at all: the solve reads the error word at its first step and the
// temporaries go back to the pool once an event after their last use has
// completed.
static int problem_create_on(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                             const int64_t* other_sizes, const double* const* factors, int32_t r,
                             int64_t q, const int32_t* kidx, const int32_t* oidx,
                             const void* vals, uint32_t flags, int mem, cudaStream_t st,
                             bool async, cphifi_problem** out) {
  if (!ctx || !out) return CPHIFI_E_INVALID_ARG;
  *out = nullptr;
  if (!kern || kern->ctx != ctx) return fail(ctx, CPHIFI_E_INVALID_ARG, "kernel of another context");
  if (d_other < 1 || d_other > 16) return fail(ctx, CPHIFI_E_INVALID_ARG, "d_other must be in [1, 16]");
  if (r < 1 || r > kMaxRank) return fail(ctx, CPHIFI_E_INVALID_ARG, "r must be in [1, 64]");
  if (q < 0 || q >= (int64_t(1) << 31)) return fail(ctx, CPHIFI_E_INVALID_ARG, "q must be in [0, 2^31)");
  if (!other_sizes || !factors) return fail(ctx, CPHIFI_E_INVALID_ARG, "null sizes or factors");
  if (q > 0 && (!kidx || !oidx || !vals)) return fail(ctx, CPHIFI_E_INVALID_ARG, "null observation list");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  std::vector<int64_t> sizes(other_sizes, other_sizes + d_other);
  double M = 1.0;
  for (int m = 0; m < d_other; ++m) {
    if (sizes[m] < 1 || sizes[m] > (int64_t(1) << 31) - 1 || !factors[m])
      return fail(ctx, CPHIFI_E_INVALID_ARG, "bad other-mode size or null factor");
    M *= (double)sizes[m];
  }
  const int n = kern->n;
  Enter guard(ctx);
  // Gather-dot/scatter decomposition: W warps, L = ceil(q / W) observations each.
  const Shapes shapes = problem_shapes(ctx, kern, n, q, r);
  const int64_t W64 = shapes.W;
  const int W = (int)W64;
  const int64_t L = std::max<int64_t>(1, (q + W - 1) / W);
  const int64_t npieces_max = (int64_t)n + W + 1;
  const int nsplit64 = shapes.s64;
  const int nsplit32 = shapes.s32;
  const int nsplitdf = shapes.sdf;
  const int nsplittc = shapes.stc;
  const int nsplit = std::max(std::max(nsplit64, nsplit32), std::max(nsplitdf, nsplittc));
  // Operator data: FP64 Zhat for the FP64 operator, hi/lo FP32 pairs for the
  // mixed modes; neither flag set means both.
  const bool need64 = (flags & CPHIFI_NEED_FP64) || !(flags & CPHIFI_NEED_LOWP);
  const bool lowp = (flags & CPHIFI_NEED_LOWP) || !(flags & CPHIFI_NEED_FP64);
  size_t need = 0, tmp_need = 0;
  problem_need(ctx, kern, d_other, sizes, r, q, flags, &need, &tmp_need);
  if (ctx->budget && ctx->in_use + need + tmp_need > ctx->budget)
    return fail(ctx, CPHIFI_E_ADMISSION, "problem footprint exceeds the HBM budget");
  auto t0 = std::chrono::steady_clock::now();
  cphifi_problem* P = new cphifi_problem();
  P->ctx = ctx;
  P->kern = kern;
  P->n = n;
  P->r = r;
  P->d_other = d_other;
  P->q = q;
  P->sizes = sizes;
  P->gamma = (double)q / ((double)n * M);
  P->st = st;
  P->nsplit64 = nsplit64;
  P->nsplit32 = nsplit32;
  P->nsplitdf = nsplitdf;
  P->nsplittc = nsplittc;
  P->ldt = kern->tc ? kern->ldt : n;
  P->nwarps = W;
  P->obs_per_warp = L;
  std::vector<std::pair<void*, size_t>> temps;
  auto tmp_alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    size_t got = 0;
    if (pool_alloc(ctx, bytes, &p, &got) != cudaSuccess) return nullptr;
    temps.push_back({p, got});
    return p;
  };
  std::vector<cudaEvent_t>* chunk_events = nullptr;  // set below when the upload is chunked
  auto bail = [&](int code, const std::string& m) {
    if (!async) {
      cudaStreamSynchronize(ctx->side);
      cudaStreamSynchronize(ctx->copy);
    }
    cudaStreamSynchronize(st);
    if (chunk_events)
      for (auto e : *chunk_events) ctx->events_free.push_back(e);
    for (auto& t : temps) pool_release(ctx, t.first, t.second);
    free_problem(P);
    delete P;
    return fail(ctx, code, m);
  };
#define PCK(...)                                                                            \
  do {                                                                                      \
    if (is_launch(#__VA_ARGS__)) P->create_launches += launch_weight(#__VA_ARGS__);         \
    cudaError_t e_ = (__VA_ARGS__);                                                         \
    if (e_ != cudaSuccess)                                                                  \
      return bail(e_ == cudaErrorMemoryAllocation ? CPHIFI_E_OOM : CPHIFI_E_DEVICE,        \
                  std::string(#__VA_ARGS__ " failed: ") + cudaGetErrorString(e_));         \
  } while (0)

  // ---- persistent arrays
  const size_t nr = (size_t)n * r;
  PCK(dalloc(P, &P->perm, q));
  PCK(dalloc(P, &P->row_ptr, n + 1));
  if (lowp) {
    PCK(dalloc(P, &P->zhi, (size_t)zhat_elems(q, r) * 2));
    P->zlo = P->zhi + 32 * (int64_t)r;
  }
  if (need64) PCK(dalloc(P, &P->z64, (size_t)zhat_elems(q, r)));
  PCK(dalloc(P, &P->warp_first, (size_t)W + 1));
  PCK(dalloc(P, &P->seg_first, n + 1));
  PCK(dalloc(P, &P->seg_count, n));
  PCK(dalloc(P, &P->seg_ticket, n));
  PCK(dalloc(P, &P->factors_dev, d_other));
  PCK(dalloc(P, &P->fhl_dev, d_other));
  PCK(dalloc(P, &P->sizes_dev, d_other));
  P->factors.resize(d_other);
  P->fhl.resize(d_other);
  for (int m = 0; m < d_other; ++m) {
    PCK(dalloc(P, &P->factors[m], (size_t)sizes[m] * r));
    PCK(dalloc(P, &P->fhl[m], (size_t)sizes[m] * r * 2));
  }
  PCK(dalloc(P, &P->V, r * r));
  PCK(dalloc(P, &P->dV, r));
  PCK(dalloc(P, &P->UV, r * r));
  PCK(dalloc(P, &P->UV32, r * r));
  PCK(dalloc(P, &P->info, 4));
  PCK(dalloc(P, &P->err, 4));
  PCK(dalloc(P, &P->Bm, nr));
  for (double** v : {&P->x, &P->res, &P->z, &P->p, &P->y, &P->bbar, &P->xh64, &P->y164,
                     &P->tmp64, &P->tmp64b, &P->D64, &P->tres})
    PCK(dalloc(P, v, nr));
  for (float** v : {&P->xh32, &P->D32, &P->Bhi, &P->Blo}) PCK(dalloc(P, v, nr));
  PCK(dalloc(P, &P->pop32, (size_t)P->ldt * r));
  PCK(dalloc(P, &P->y132, (size_t)P->ldt * r));
  PCK(cudaMemsetAsync(P->pop32, 0, (size_t)P->ldt * r * sizeof(float), st));
  PCK(cudaMemsetAsync(P->y132, 0, (size_t)P->ldt * r * sizeof(float), st));
  if (kern->tc) {
    PCK(dalloc(P, &P->pop16, (size_t)P->ldt * r));
    PCK(dalloc(P, &P->y116, (size_t)P->ldt * r));
    for (float** v : {&P->poph, &P->popl, &P->y1h, &P->y1l}) {
      PCK(dalloc(P, v, (size_t)P->ldt * r));
      PCK(cudaMemsetAsync(*v, 0, (size_t)P->ldt * r * sizeof(float), st));
    }
    PCK(dalloc(P, &P->tc_err, 1));
    PCK(cudaMemsetAsync(P->tc_err, 0, sizeof(int), st));
    const uint32_t np = (uint32_t)tc_pad_cols(r);
    PCK(tc_make_map(&P->mBpf, P->pop32, false, n, r, P->ldt * 4, np));
    PCK(tc_make_map(&P->mByf, P->y132, false, n, r, P->ldt * 4, np));
    PCK(tc_make_map(&P->mBpb, P->pop16, true, n, r, P->ldt * 2, np));
    PCK(tc_make_map(&P->mByb, P->y116, true, n, r, P->ldt * 2, np));
    PCK(tc_make_map(&P->mBph, P->poph, false, n, r, P->ldt * 4, np));
    PCK(tc_make_map(&P->mBpl, P->popl, false, n, r, P->ldt * 4, np));
    PCK(tc_make_map(&P->mByh, P->y1h, false, n, r, P->ldt * 4, np));
    PCK(tc_make_map(&P->mByl, P->y1l, false, n, r, P->ldt * 4, np));
    if (kern->oz) {
      const size_t cnt = (size_t)7 * 64 * P->ldt;  // 7 slices of 64 rows (r padded)
      PCK(dalloc(P, &P->ozb, cnt));
      PCK(cudaMemsetAsync(P->ozb, 0, cnt * sizeof(__nv_bfloat16), st));
      PCK(dalloc(P, &P->ozce, 64));
      PCK(oz_make_b_map(P->ozb, n, r, P->ldt, &P->mOzb));
    }
  }
  PCK(dalloc(P, (double**)&P->cpart, (size_t)nsplit * nr));
  PCK(dalloc(P, &P->red.partials, (size_t)kRedMaxBlocks * kRedSlots));
  PCK(dalloc(P, &P->red.ticket, 4));
  PCK(dalloc(P, &P->s, 1));
  PCK(dalloc(P, &P->s2, 1));
  PCK(cudaMemsetAsync(P->red.ticket, 0, 4 * sizeof(unsigned), st));
  // pinned: the scalars, then the tensor-core error word
  {
    void* h = nullptr;
    PCK(pinned_get(ctx, &h));
    P->hs = (DevScalars*)h;
  }
  for (auto& e : P->ev) PCK(event_get(ctx, &e));
  PCK(cudaMemsetAsync(P->seg_ticket, 0, n * sizeof(unsigned), st));
  PCK(dalloc(P, &P->wctr, 2));
  PCK(cudaMemsetAsync(P->wctr, 0, 2 * sizeof(unsigned), st));
  PCK(cudaMemsetAsync(P->err, 0, sizeof(int), st));
  PCK(cudaMemsetAsync(P->info, 0, sizeof(int), st));

  // ---- factors
  PCK(cudaMemcpyAsync(P->factors_dev, P->factors.data(), d_other * sizeof(double*),
                      cudaMemcpyHostToDevice, st));
  PCK(cudaMemcpyAsync(P->fhl_dev, P->fhl.data(), d_other * sizeof(float*),
                      cudaMemcpyHostToDevice, st));
  PCK(cudaMemcpyAsync(P->sizes_dev, sizes.data(), d_other * sizeof(int64_t),
                      cudaMemcpyHostToDevice, st));
  for (int m = 0; m < d_other; ++m) {
    PCK(upload(P->factors[m], factors[m], (size_t)sizes[m] * r * sizeof(double), mem, st));
    PCK(launch_validate_dense(P->factors[m], sizes[m] * r, P->err, st));
    PCK(launch_split_rows_df(P->factors[m], sizes[m], r, P->fhl[m], st));
  }

  // ---- Gram V (§3) and eig(V) (Eq. eigV): they need only the factors.  A
  // synchronous creation runs them on the context's second stream, under the
  // observation passes below (whose blocks draw their work from a counter, so
  // the SM that the one-block eigensolver holds only lowers their rate by a
  // block's share); a submitted request, already on a stream of its own among
  // others, runs them in order.
  cudaStream_t gst = async ? st : ctx->side;
  if (!async) {
    PCK(cudaEventRecord(ctx->ev_fork, st));
    PCK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  }
  PCK(launch_gram(P->factors_dev, P->sizes_dev, d_other, r, P->V, gst));
  PCK(launch_jacobi_eig(P->V, r, P->dV, P->UV, 60, P->info, gst));
  PCK(launch_convert<double, float>(P->UV, P->UV32, (int64_t)r * r, gst));
  if (!async) PCK(cudaEventRecord(ctx->ev_join, ctx->side));

  // ---- observations: copy, validate, sort by kernel index
  const bool sorted_in = (flags & CPHIFI_OBS_SORTED) != 0;
  uint32_t* keys = sorted_in ? nullptr : (uint32_t*)tmp_alloc((size_t)q * sizeof(uint32_t));
  int32_t* oidx_d = nullptr;
  const double* vals_d = nullptr;
  const int32_t* kidx_d = nullptr;
  const bool vals32 = (flags & CPHIFI_VALS_F32) != 0;
  const size_t vbytes = (size_t)q * (vals32 ? sizeof(float) : sizeof(double));
  if (!sorted_in && !keys) return bail(CPHIFI_E_OOM, "temporary allocation failed");
  const void* vsrc = vals;  // the values on the device, in the caller's type
  // Host inputs of a large sorted problem, synchronous creation: the kernel
  // indices go first (the row pointer and the pieces need them); the other
  // indices and the values follow in kUploadChunks chunks on the copy stream,
  // and the Zhat pass runs chunk by chunk behind them (the host link, ~210
  // GB/s, then overlaps the pass instead of preceding it).
  const bool pipelined = mem == CPHIFI_MEM_HOST && sorted_in && !async && q >= kPipelineMinQ;
  std::vector<cudaEvent_t> chunk_ready;
  chunk_events = &chunk_ready;
  if (mem == CPHIFI_MEM_DEVICE) {
    oidx_d = (int32_t*)oidx;
    kidx_d = kidx;
  } else {
    oidx_d = (int32_t*)tmp_alloc((size_t)q * d_other * sizeof(int32_t));
    void* v = tmp_alloc(vbytes);
    int32_t* k = (int32_t*)tmp_alloc((size_t)q * sizeof(int32_t));
    if (!oidx_d || !v || !k) return bail(CPHIFI_E_OOM, "temporary allocation failed");
    PCK(upload(k, kidx, (size_t)q * sizeof(int32_t), mem, st));
    if (!pipelined) {
      PCK(upload(oidx_d, oidx, (size_t)q * d_other * sizeof(int32_t), mem, st));
      PCK(upload(v, vals, vbytes, mem, st));
    }
    vsrc = v;
    kidx_d = k;
  }
  double* v64 = nullptr;
  if (vals32 && q > 0) {  // FP32 values are widened to FP64 once, on the device
    v64 = (double*)tmp_alloc((size_t)q * sizeof(double));
    if (!v64) return bail(CPHIFI_E_OOM, "temporary allocation failed");
    if (!pipelined) PCK(launch_convert<float, double>((const float*)vsrc, v64, q, st));
    vals_d = v64;
  } else {
    vals_d = (const double*)vsrc;
  }
  if (pipelined) {
    int64_t W2 = 0, L2 = 0;
    zhat_ranges(ctx->num_sms, n, q, &W2, &L2);
    cudaStream_t cs = ctx->copy;
    PCK(cudaEventRecord(ctx->ev_in, st));  // after the caller's work on its stream
    PCK(cudaStreamWaitEvent(cs, ctx->ev_in, 0));
    const size_t es = vals32 ? sizeof(float) : sizeof(double);
    for (int c = 0; c < kUploadChunks; ++c) {
      int64_t w0, w1, o0, o1;
      zhat_chunk(W2, L2, q, kUploadChunks, c, &w0, &w1, &o0, &o1);
      cudaEvent_t ev = nullptr;
      PCK(event_get(ctx, &ev));
      chunk_ready.push_back(ev);
      if (o1 > o0) {
        PCK(upload(oidx_d + o0 * d_other, oidx + o0 * d_other,
                   (size_t)(o1 - o0) * d_other * sizeof(int32_t), mem, cs));
        PCK(upload((char*)vsrc + o0 * es, (const char*)vals + o0 * es, (size_t)(o1 - o0) * es,
                   mem, cs));
        if (vals32)
          PCK(launch_convert<float, double>((const float*)vsrc + o0, v64 + o0, o1 - o0, cs));
      }
      PCK(cudaEventRecord(ev, cs));
    }
  }
  // kernel indices here (the sort and the pieces use them); the other
  // indices and the values are checked by the Zhat build below
  PCK(launch_validate_kidx(kidx_d, q, n, sorted_in, P->err, st));
  if (!sorted_in)
    PCK(cudaMemcpyAsync(keys, kidx_d, (size_t)q * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  // sorted keys: the validated (non-negative) kernel indices themselves
  const uint32_t* skeys = sorted_in ? reinterpret_cast<const uint32_t*>(kidx_d) : keys;
  PCK(launch_iota(P->perm, q, st));
  // No host wait from here on: the kernels after the validation are gated on
  // the error word, which a synchronous creation reads once at the end.
  int herr = 0;
  const int* gate = P->err;
  if (!sorted_in && q > 1) {
    void* rtmp = tmp_alloc(radix_sort_tmp_bytes(q));
    if (!rtmp) return bail(CPHIFI_E_OOM, "temporary allocation failed");
    PCK(radix_sort_pairs(keys, P->perm, q, bits_for(n), rtmp, st));
  }
  PCK(launch_row_ptr(skeys, q, n, P->row_ptr, st));
  // ---- pieces
  {
    void* stmp = tmp_alloc(exclusive_scan_tmp_bytes(n));
    if (!stmp) return bail(CPHIFI_E_OOM, "temporary allocation failed");
    PCK(launch_piece_counts(P->row_ptr, n, L, P->seg_count, gate, st));
    PCK(exclusive_scan_i32(P->seg_count, P->seg_first, n, stmp, exclusive_scan_tmp_bytes(n), st));
    int np = 0;
    np = q > 0 ? (int)npieces_max : 0;  // the exact count stays on the device
    P->npieces = np;
    PCK(dalloc(P, &P->pseg, np));
    PCK(dalloc(P, &P->pbeg, np));
    PCK(dalloc(P, &P->pend, np));
    PCK(dalloc(P, (double**)&P->gds_partial, (size_t)np * 64));
    PCK(launch_piece_fill(P->row_ptr, n, L, P->seg_first, P->seg_count, P->pseg, P->pbeg,
                          P->pend, gate, st));
    PCK(launch_warp_first(P->pbeg, np, P->seg_first + n, L, W, P->warp_first, gate, st));
  }

  // ---- Zhat and the right-hand side MTTKRP
  {
    const cudaError_t ez = zhat_and_rhs(P, (flags & CPHIFI_OBS_SORTED) ? nullptr : P->perm,
                                        oidx_d, vals_d, gate, tmp_alloc, st,
                                        pipelined ? &chunk_ready : nullptr);
    if (ez == cudaErrorMemoryAllocation) return bail(CPHIFI_E_OOM, "temporary allocation failed");
    PCK(ez);
  }
  if (flags & CPHIFI_KEEP_OBS) {
    P->keep_obs = true;
    PCK(dalloc(P, &P->kidx_s, (size_t)q));
    PCK(dalloc(P, &P->oidx_s, (size_t)q * d_other));
    PCK(dalloc(P, &P->vals_s, (size_t)q));
    PCK(dalloc(P, &P->Ak, (size_t)n * r));
    PCK(dalloc(P, &P->fit2, 2));
    PCK(dalloc(P, &P->nfail, 4));
    P->perm_m.assign(d_other, nullptr);
    P->rowp_m.assign(d_other, nullptr);
    PCK(launch_keep_obs(q, d_other, skeys, (flags & CPHIFI_OBS_SORTED) ? nullptr : P->perm,
                        oidx_d, vals_d, P->kidx_s, P->oidx_s, P->vals_s, gate, st));
  }
  if (!async) PCK(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  if (async) {
    cudaEvent_t ev = nullptr;
    PCK(event_get(ctx, &ev));
    PCK(cudaEventRecord(ev, st));
    for (auto& t : temps) ctx->deferred_bytes += t.second;
    ctx->deferred.push_back({ev, std::move(temps)});
    temps.clear();
  } else {
    PCK(cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PCK(cudaStreamSynchronize(st));
    for (auto e : chunk_ready) ctx->events_free.push_back(e);
    chunk_ready.clear();
    if (herr) return bail(CPHIFI_E_INVALID_ARG, input_error_text(herr));
    // the temporaries are free to reuse only after the work (synchronized above)
    for (auto& t : temps) pool_release(ctx, t.first, t.second);
    temps.clear();
  }
  (void)t0;
  *out = P;
  return CPHIFI_OK;
#undef PCK
}

extern "C" int cphifi_problem_create(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                                     const int64_t* other_sizes, const double* const* factors,
                                     int32_t r, int64_t q, const int32_t* kidx,
                                     const int32_t* oidx, const void* vals, uint32_t flags,
                                     int mem, cphifi_problem** out) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  return problem_create_on(ctx, kern, d_other, other_sizes, factors, r, q, kidx, oidx, vals,
                           flags, mem, ctx->stream, /*async=*/false, out);
}

extern "C" int cphifi_problem_destroy(cphifi_problem* P) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(P->st);
  free_problem(P);
  cudaSetDevice(prev);
  delete P;
  return CPHIFI_OK;
}

extern "C" size_t cphifi_problem_bytes(const cphifi_problem* P) { return P ? P->bytes : 0; }

// ------------------------------------------------------------- solve ------
namespace {

bool is_lowp(int prec) {
  return prec == CPHIFI_MIXED_FP32 || prec == CPHIFI_MIXED_TF32 || prec == CPHIFI_MIXED_BF16 ||
         prec == CPHIFI_MIXED_TF32X3 || prec == CPHIFI_MIXED_BF16X3;
}
bool is_tc(int prec) {
  return prec == CPHIFI_MIXED_TF32 || prec == CPHIFI_MIXED_BF16 || prec == CPHIFI_MIXED_TF32X3;
}

struct Launcher {
  cphifi_problem* P;
  cudaStream_t st;
  Timer* tm;
  int64_t launches = 0;
  // 0: every product streams Zhat; 1: the iteration operator (CM_APPLY)
  // applies the per-index Gram blocks instead; 2: the checks as well.
  int gram = 0;
  bool gram_for(int mode) const { return gram == 2 || (gram == 1 && mode == CM_APPLY); }

  PieceList pieces() const {
    return PieceList{P->pseg, P->pbeg, P->pend, P->seg_first, P->seg_count, P->seg_ticket,
                     P->warp_first, P->npieces, P->nwarps, P->wctr};
  }
  int64_t split_stride() const { return (int64_t)P->n * P->r; }

  // out = U_K diag(scale) Bx  (a_trans: U_K itself), FP64, into out (n x r)
  // cat: 0 untimed, 1 operator arithmetic of the PCG iteration, 2 FP64
  // true-residual arithmetic of the mixed solve.
  cudaError_t gemm64(bool a_trans, const double* scale, const double* B, double* out_part,
                     const DevScalars* skip, int cat) {
    cudaEvent_t b = cat && tm ? tm->begin() : nullptr;
    cudaError_t e = launch_gemm_skinny<double, double>(P->kern->UK64, P->n, a_trans, scale, B, P->n,
                                                       out_part, P->n, split_stride(), P->n, P->r,
                                                       P->nsplit64, skip, st);
    if (cat && tm) tm->end(b, cat == 1 ? tm->gemm : tm->gemm64);
    ++launches;
    return e;
  }
  // FP32 SIMT product; B has leading dimension ldb.
  cudaError_t gemm32(bool a_trans, const double* scale, const float* B, int64_t ldb,
                     float* out_part, const DevScalars* skip) {
    cudaEvent_t b = tm ? tm->begin() : nullptr;
    cudaError_t e = launch_gemm_skinny<float, float>(P->kern->UK32, P->n, a_trans, scale, B, ldb,
                                                     out_part, P->n, split_stride(), P->n, P->r,
                                                     P->nsplit32, skip, st);
    if (tm) tm->end(b, tm->gemm);
    ++launches;
    return e;
  }
  // Tensor-core product (tcgen05): g1 = U_K pop, else U_K' y1; TF32, BF16,
  // or the 3-term split TF32 (x3).
  cudaError_t gemm_tc(bool g1, bool bf16, bool x3, float* out_part, const DevScalars* skip) {
    const cphifi_kernel* K = P->kern;
    const CUtensorMap* ma;
    const CUtensorMap* mb;
    const CUtensorMap* mal = nullptr;
    const CUtensorMap* mbl = nullptr;
    if (x3) {
      ma = g1 ? &K->mA1h : &K->mA2h;
      mal = g1 ? &K->mA1l : &K->mA2l;
      mb = g1 ? &P->mBph : &P->mByh;
      mbl = g1 ? &P->mBpl : &P->mByl;
    } else {
      ma = g1 ? (bf16 ? &K->mA1b : &K->mA1f) : (bf16 ? &K->mA2b : &K->mA2f);
      mb = g1 ? (bf16 ? &P->mBpb : &P->mBpf) : (bf16 ? &P->mByb : &P->mByf);
    }
    cudaEvent_t b = tm ? tm->begin() : nullptr;
    cudaError_t e = launch_tc_gemm(bf16, *ma, *mb, mal, mbl, out_part, P->n, split_stride(), P->n,
                                   P->r, P->nsplittc, skip, P->tc_err, st);
    if (tm) tm->end(b, tm->gemm);
    ++launches;
    return e;
  }
  // FP64-accurate product without the FP64 units: out_part gets the partial
  // products of op(U_K) diag(scale) B over nsplitdf splits, from the BF16
  // slices on the tensor cores (oz_gemm.cu) when the kernel has them, else in
  // double-float arithmetic on the FP32 units.
  // op(U_K) diag(scale) B from `slices` BF16 slices of each operand (the
  // kernel's slices must exist), timed as an operator product.
  cudaError_t gemm_oz(bool a_trans, const double* scale, const double* B, double* out_part,
                      const DevScalars* skip, int slices) {
    const cphifi_kernel* K = P->kern;
    cudaError_t e = launch_oz_b(B, scale, P->n, P->r, P->n, P->ldt, P->ozb, P->ozce, skip, st);
    ++launches;
    if (e != cudaSuccess) return e;
    cudaEvent_t b = tm ? tm->begin() : nullptr;
    e = launch_oz_gemm(a_trans ? K->mOz1 : K->mOz2, a_trans ? K->oze : K->oze + P->n, P->mOzb,
                       P->ozce, out_part, P->n, split_stride(), P->n, P->r, P->nsplitdf, skip,
                       P->tc_err, st, slices);
    if (tm) tm->end(b, tm->gemm);
    ++launches;
    return e;
  }
  cudaError_t gemm_df(bool a_trans, const double* scale, const double* B, double* out_part,
                      const DevScalars* skip, int cat) {
    if (P->ozb) {  // tensor cores, from BF16 slices of both operands
      const cphifi_kernel* K = P->kern;
      cudaError_t e = launch_oz_b(B, scale, P->n, P->r, P->n, P->ldt, P->ozb, P->ozce, skip, st);
      ++launches;
      if (e != cudaSuccess) return e;
      cudaEvent_t b = cat && tm ? tm->begin() : nullptr;
      e = launch_oz_gemm(a_trans ? K->mOz1 : K->mOz2, a_trans ? K->oze : K->oze + P->n, P->mOzb,
                         P->ozce, out_part, P->n, split_stride(), P->n, P->r, P->nsplitdf, skip,
                         P->tc_err, st);
      if (cat && tm) tm->end(b, cat == 1 ? tm->gemm : tm->gemm64);
      ++launches;
      return e;
    }
    cudaError_t e = launch_split_df(B, scale, P->n, (int64_t)P->n * P->r, P->Bhi, P->Blo, st);
    ++launches;
    if (e != cudaSuccess) return e;
    cudaEvent_t b = cat && tm ? tm->begin() : nullptr;
    e = launch_gemm_df(P->kern->UK32, P->kern->UKlo, P->n, a_trans, P->Bhi, P->Blo, P->n,
                       out_part, P->n, split_stride(), P->n, P->r, P->nsplitdf, skip, st);
    if (cat && tm) tm->end(b, cat == 1 ? tm->gemm : tm->gemm64);
    ++launches;
    return e;
  }
  // ns: number of split partials in C (0 = the FP64/FP32 product default).
  template <typename TC, typename TO>
  cudaError_t combine(int mode, const TC* C, const double* V, const double* Bv, TO* out,
                      DevScalars* s, const DevScalars* skip, int ns = 0) {
    ++launches;
    if (ns == 0) ns = sizeof(TC) == 8 ? P->nsplit64 : P->nsplit32;
    return launch_combine<TC, TO>(mode, C, split_stride(), ns, P->n, P->r, P->kern->dK, V,
                                  Bv, out, s, P->red, skip, st);
  }
  // Gather-dot/scatter in the three arithmetics (cat as for the products).
  cudaError_t gds32(const float* Xh, float* Y, const DevScalars* skip, int cat,
                    int64_t yld = 0) {
    cudaEvent_t b = (cat && tm) ? tm->begin() : nullptr;
    cudaError_t e = launch_gds_f32(pieces(), P->zhi, P->r, Xh, P->n, (float*)P->gds_partial, Y,
                                   yld ? yld : P->n, skip, st);
    if (cat && tm) tm->end(b, cat == 1 ? tm->gds : tm->gds64);
    ++launches;
    return e;
  }
  cudaError_t gds64(const double* Xh, double* Y, const DevScalars* skip, int cat) {
    cudaEvent_t b = (cat && tm) ? tm->begin() : nullptr;
    cudaError_t e = launch_gds_f64(pieces(), P->z64, P->r, Xh, P->n, (double*)P->gds_partial, Y,
                                   P->n, skip, st);
    if (cat && tm) tm->end(b, cat == 1 ? tm->gds : tm->gds64);
    ++launches;
    return e;
  }
  cudaError_t gdsdf(const double* Xh, double* Y, const DevScalars* skip, int cat) {
    cudaEvent_t b = (cat && tm) ? tm->begin() : nullptr;
    cudaError_t e = launch_gds_df(pieces(), P->zhi, P->zlo, P->r, Xh, P->n,
                                  (double*)P->gds_partial, Y, P->n, skip, st);
    if (cat && tm) tm->end(b, cat == 1 ? tm->gds : tm->gds64);
    ++launches;
    return e;
  }

  // Yhat1 from the per-index Gram blocks (Eq. yhat1 with the sum over the
  // observations done once): FP32 blocks, or the FP64-accurate ones.
  cudaError_t gram32(const float* Xh, float* Y, const DevScalars* skip, int cat,
                     int64_t yld = 0) {
    cudaEvent_t b = (cat && tm) ? tm->begin() : nullptr;
    cudaError_t e = launch_gram_apply_f32(P->C32, P->n, P->r, Xh, P->n, Y, yld ? yld : P->n,
                                          skip, st);
    if (cat && tm) tm->end(b, cat == 1 ? tm->gds : tm->gds64);
    ++launches;
    return e;
  }
  cudaError_t gram64(const double* Xh, double* Y, const DevScalars* skip, int cat) {
    cudaEvent_t b = (cat && tm) ? tm->begin() : nullptr;
    cudaError_t e = launch_gram_apply_f64(P->C64, P->n, P->r, Xh, P->n, Y, P->n, skip, st);
    if (cat && tm) tm->end(b, cat == 1 ? tm->gds : tm->gds64);
    ++launches;
    return e;
  }

  // FP64 operator in the eigenbasis: out = Abar xin (mode CM_APPLY) or the
  // true residual res = bbar - Abar xin (mode CM_RESID).
  cudaError_t op64(int mode, const double* xin, double* out, DevScalars* s,
                   const DevScalars* skip, int cat) {
    double* Cp = (double*)P->cpart;
    cudaError_t e;
    if ((e = gemm64(true, P->kern->dK, xin, Cp, skip, cat)) != cudaSuccess) return e;
    if ((e = combine<double, double>(CM_STORE, Cp, nullptr, nullptr, P->xh64, s, skip)) != cudaSuccess) return e;
    if ((e = (gram_for(mode) && P->c64_ok) ? gram64(P->xh64, P->y164, skip, cat)
                                           : gds64(P->xh64, P->y164, skip, cat)) != cudaSuccess)
      return e;
    if ((e = gemm64(false, nullptr, P->y164, Cp, skip, cat)) != cudaSuccess) return e;
    return combine<double, double>(mode, Cp, xin, P->bbar, out, s, skip);
  }
  // The same operator FP64-accurate without the FP64 units (double-float
  // gather/scatter, split-operand or double-float products).
  cudaError_t opdf(int mode, const double* xin, double* out, DevScalars* s,
                   const DevScalars* skip, int cat) {
    double* Cp = (double*)P->cpart;
    const int ns = P->nsplitdf;
    cudaError_t e;
    if ((e = gemm_df(true, P->kern->dK, xin, Cp, skip, cat)) != cudaSuccess) return e;
    if ((e = combine<double, double>(CM_STORE, Cp, nullptr, nullptr, P->xh64, s, skip, ns)) != cudaSuccess) return e;
    if ((e = (gram_for(mode) && P->c64_ok) ? gram64(P->xh64, P->y164, skip, cat)
                                           : gdsdf(P->xh64, P->y164, skip, cat)) != cudaSuccess)
      return e;
    if ((e = gemm_df(false, nullptr, P->y164, Cp, skip, cat)) != cudaSuccess) return e;
    return combine<double, double>(mode, Cp, xin, P->bbar, out, s, skip, ns);
  }
  // Low-precision operator (mixed modes): pop32 (and pop16 for BF16) hold
  // D_K xin in the operand type; FP32 SIMT products, or tcgen05 TF32/BF16.
  cudaError_t op_lowp(int prec, const double* xin, double* out, DevScalars* s,
                      const DevScalars* skip) {
    if (prec == CPHIFI_MIXED_BF16X3) return op_bf16x3(xin, out, s, skip);
    const bool x3 = prec == CPHIFI_MIXED_TF32X3;
    const bool tc = prec == CPHIFI_MIXED_TF32 || prec == CPHIFI_MIXED_BF16 || x3;
    const bool bf = prec == CPHIFI_MIXED_BF16;
    float* Cp = (float*)P->cpart;
    const int ns = tc ? P->nsplittc : P->nsplit32;
    cudaError_t e;
    if (x3) {
      ++launches;
      if ((e = launch_tf32_split_block(P->pop32, P->ldt, P->n, (int64_t)P->n * P->r, P->poph,
                                       P->popl, P->ldt, skip, st)) != cudaSuccess)
        return e;
    }
    e = tc ? gemm_tc(true, bf, x3, Cp, skip) : gemm32(true, nullptr, P->pop32, P->ldt, Cp, skip);
    if (e != cudaSuccess) return e;
    if ((e = combine<float, float>(CM_STORE, Cp, nullptr, nullptr, P->xh32, s, skip, ns)) != cudaSuccess) return e;
    // Yhat1 with leading dimension ldt (the product operand), dense for the
    // BF16 conversion that feeds the BF16 product
    const int64_t yld = bf ? P->n : P->ldt;
    if ((e = (gram >= 1 && P->c32_ok) ? gram32(P->xh32, P->y132, skip, 1, yld)
                                      : gds32(P->xh32, P->y132, skip, 1, yld)) != cudaSuccess)
      return e;
    if (bf) {
      ++launches;
      if ((e = launch_scale_to<float, __nv_bfloat16>(P->y132, nullptr, P->n, (int64_t)P->n * P->r,
                                                     P->y116, P->ldt, st)) != cudaSuccess)
        return e;
    }
    if (x3) {
      ++launches;
      if ((e = launch_tf32_split_block(P->y132, P->ldt, P->n, (int64_t)P->n * P->r, P->y1h,
                                       P->y1l, P->ldt, skip, st)) != cudaSuccess)
        return e;
    }
    e = tc ? gemm_tc(false, bf, x3, Cp, skip) : gemm32(false, nullptr, P->y132, P->ldt, Cp, skip);
    if (e != cudaSuccess) return e;
    return combine<float, double>(CM_APPLY, Cp, xin, nullptr, out, s, skip, ns);
  }
  // Low-precision operator from 3 BF16 slices per operand on the tensor
  // cores: Xhat = U_K (D_K xin) into FP64 partials, summed and rounded to
  // FP32 for the FP32 gather-dot/scatter, then U_K' Yhat1 from Yhat1 widened
  // to FP64 (its slices are cut from the FP64 values).
  cudaError_t op_bf16x3(const double* xin, double* out, DevScalars* s, const DevScalars* skip) {
    double* Cp = (double*)P->cpart;
    const int ns = P->nsplitdf;
    cudaError_t e;
    if ((e = gemm_oz(true, P->kern->dK, xin, Cp, skip, 3)) != cudaSuccess) return e;
    if ((e = combine<double, float>(CM_STORE, Cp, nullptr, nullptr, P->xh32, s, skip, ns)) != cudaSuccess) return e;
    if ((e = (gram >= 1 && P->c32_ok) ? gram32(P->xh32, P->y132, skip, 1, P->n)
                                      : gds32(P->xh32, P->y132, skip, 1, P->n)) != cudaSuccess)
      return e;
    ++launches;
    if ((e = launch_convert<float, double>(P->y132, P->y164, (int64_t)P->n * P->r, st)) != cudaSuccess)
      return e;
    if ((e = gemm_oz(false, nullptr, P->y164, Cp, skip, 3)) != cudaSuccess) return e;
    return combine<double, double>(CM_APPLY, Cp, xin, nullptr, out, s, skip, ns);
  }
  // FP64-accurate operator of the given arithmetic (mode: CM_APPLY / CM_RESID).
  cudaError_t opwide(bool emulated, int mode, const double* xin, double* out, DevScalars* s,
                     const DevScalars* skip, int cat) {
    return emulated ? opdf(mode, xin, out, s, skip, cat) : op64(mode, xin, out, s, skip, cat);
  }
  // out = D_K U_K' B (emulated: the FP64-accurate product of gemm_df) with
  // ||out||^2 -> bb
  // when norm is set; the right-hand side and the start transform.
  cudaError_t utb(bool emulated, int mode, const double* B, double* out, DevScalars* s) {
    double* Cp = (double*)P->cpart;
    cudaError_t e = emulated ? gemm_df(false, nullptr, B, Cp, nullptr, 0)
                             : gemm64(false, nullptr, B, Cp, nullptr, 0);
    if (e != cudaSuccess) return e;
    return combine<double, double>(mode, Cp, nullptr, nullptr, out, s, nullptr,
                                   emulated ? P->nsplitdf : P->nsplit64);
  }
  // out = U_K x (emulated: the FP64-accurate product of gemm_df).
  cudaError_t ux(bool emulated, const double* x, double* out, DevScalars* s) {
    double* Cp = (double*)P->cpart;
    cudaError_t e = emulated ? gemm_df(true, nullptr, x, Cp, nullptr, 0)
                             : gemm64(true, nullptr, x, Cp, nullptr, 0);
    if (e != cudaSuccess) return e;
    return combine<double, double>(CM_STORE, Cp, nullptr, nullptr, out, s, nullptr,
                                   emulated ? P->nsplitdf : P->nsplit64);
  }

  // The operand of the next low-precision product: pop = D_K p (+ BF16 copy).
  cudaError_t pupdate_lowp(int prec) {
    ++launches;
    if (prec == CPHIFI_MIXED_BF16X3)  // the product slices p itself: no FP32 operand copy
      return launch_pupdate<float>(P->n, P->r, P->z, P->p, nullptr, nullptr, P->n, nullptr, P->s,
                                   st);
    return launch_pupdate<float>(P->n, P->r, P->z, P->p, P->pop32, P->kern->dK, P->ldt,
                                 prec == CPHIFI_MIXED_BF16 ? P->pop16 : nullptr, P->s, st);
  }

  // One PCG iteration (operator, update + preconditioner, direction).  The
  // mixed modes use the low-precision operator and an FP32 preconditioner;
  // FP64 and FP64_EMULATED the FP64-accurate operator.
  cudaError_t iteration(int prec) {
    DevScalars* s = P->s;
    const bool lowop = is_lowp(prec);
    cudaError_t e;
    ++launches;
    if (lowop) {
      if ((e = op_lowp(prec, P->p, P->y, s, s)) != cudaSuccess) return e;
      if ((e = launch_update_precond<float>(UP_ITER, P->n, P->r, P->x, P->res, P->p, P->y, P->z,
                                            P->UV32, P->D32, s, P->red, st)) != cudaSuccess)
        return e;
      return pupdate_lowp(prec);
    }
    if ((e = opwide(prec == CPHIFI_FP64_EMULATED, CM_APPLY, P->p, P->y, s, s, 1)) != cudaSuccess)
      return e;
    if ((e = launch_update_precond<double>(UP_ITER, P->n, P->r, P->x, P->res, P->p, P->y, P->z,
                                           P->UV, P->D64, s, P->red, st)) != cudaSuccess)
      return e;
    ++launches;
    return launch_pupdate<double>(P->n, P->r, P->z, P->p, nullptr, nullptr, P->n, nullptr, s, st);
  }

  // FP64-accurate true residual of x, then a restart from it (p = z).
  cudaError_t true_residual_restart(int prec) {
    DevScalars* s = P->s;
    cudaError_t e;
    if ((e = opwide(prec != CPHIFI_FP64, CM_RESID, P->x, P->res, s, nullptr,
                    is_lowp(prec) ? 2 : 1)) != cudaSuccess)
      return e;
    return restart(prec);
  }
  // Mixed modes: FP64-accurate true residual into tres (convergence decided
  // on it); the recurrence is left as it is.
  cudaError_t true_residual_check(int prec) {
    return opwide(true, CM_TRUE, P->x, P->tres, P->s, nullptr, 2);
  }
  // The checked true residual replaces the recurrence residual; restart.
  cudaError_t adopt_restart(int prec) {
    ++launches;
    cudaError_t e = launch_adopt_residual(P->tres, P->res, (int64_t)P->n * P->r, P->s, st);
    if (e != cudaSuccess) return e;
    return restart(prec);
  }
  cudaError_t restart(int prec) {
    DevScalars* s = P->s;
    cudaError_t e;
    ++launches;
    if (is_lowp(prec)) {
      if ((e = launch_update_precond<float>(UP_RESTART, P->n, P->r, P->x, P->res, P->p, P->y,
                                            P->z, P->UV32, P->D32, s, P->red, st)) != cudaSuccess)
        return e;
      return pupdate_lowp(prec);
    }
    if ((e = launch_update_precond<double>(UP_RESTART, P->n, P->r, P->x, P->res, P->p, P->y, P->z,
                                           P->UV, P->D64, s, P->red, st)) != cudaSuccess)
      return e;
    ++launches;
    return launch_pupdate<double>(P->n, P->r, P->z, P->p, nullptr, nullptr, P->n, nullptr, s, st);
  }
};

int check_params(cphifi_ctx* ctx, const cphifi_params* prm) {
  if (!prm) return fail(ctx, CPHIFI_E_INVALID_ARG, "null params");
  if (!(prm->lambda >= 0.0) || !std::isfinite(prm->lambda))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "lambda must be finite and >= 0");
  if (!(prm->rho > 0.0) || !std::isfinite(prm->rho))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "rho must be finite and > 0");
  if (!(prm->tol > 0.0) || !std::isfinite(prm->tol))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "tol must be finite and > 0");
  if (prm->max_iter < 0) return fail(ctx, CPHIFI_E_INVALID_ARG, "max_iter must be >= 0");
  if (prm->precision < CPHIFI_FP64 || prm->precision > CPHIFI_MIXED_BF16X3)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "unknown precision");
  if (prm->gram < 0 || prm->gram > 2) return fail(ctx, CPHIFI_E_INVALID_ARG, "gram must be 0, 1 or 2");
  return CPHIFI_OK;
}

// The mixed and double-float arithmetics read Zhat as hi/lo FP32 pairs; the
// FP64 operator reads FP64.  A problem built for one gets the other on first
// use (one elementwise pass).
int ensure_lowp(cphifi_problem* P) {
  cphifi_ctx* ctx = P->ctx;
  if (P->zhi) return CPHIFI_OK;
  const size_t elems = (size_t)zhat_elems(P->q, P->r);
  if (ctx->budget && ctx->in_use + 2 * elems * sizeof(float) > ctx->budget)
    return fail(ctx, CPHIFI_E_ADMISSION, "hi/lo operator data exceeds the HBM budget");
  CK(dalloc(P, &P->zhi, elems * 2));
  P->zlo = P->zhi + 32 * (int64_t)P->r;
  CK(launch_zhat_split(P->z64, P->q, P->r, P->zhi, P->st));
  return CPHIFI_OK;
}

int ensure_fp64(cphifi_problem* P) {
  cphifi_ctx* ctx = P->ctx;
  if (P->z64) return CPHIFI_OK;
  const size_t elems = (size_t)zhat_elems(P->q, P->r);
  if (ctx->budget && ctx->in_use + elems * sizeof(double) > ctx->budget)
    return fail(ctx, CPHIFI_E_ADMISSION, "FP64 operator data exceeds the HBM budget");
  CK(dalloc(P, &P->z64, elems));
  CK(launch_zhat_join(P->zhi, P->q, P->r, P->z64, P->st));
  return CPHIFI_OK;
}

// The per-index Gram blocks (FP32 and/or FP64-accurate) on the problem's
// stream, built once and kept.  The FP32 blocks come from Zhat's hi parts;
// the FP64-accurate ones from the hi/lo pair, or from the FP64 copy when the
// problem has only that.
int ensure_grams(cphifi_problem* P, bool want32, bool want64) {
  cphifi_ctx* ctx = P->ctx;
  if ((!want32 || P->c32_ok) && (!want64 || P->c64_ok)) return CPHIFI_OK;
  if (want32 || !P->z64) {
    const int rc = ensure_lowp(P);
    if (rc != CPHIFI_OK) return rc;
  }
  const int n = P->n, r = P->r;
  const int64_t q = P->q;
  const size_t rr = (size_t)r * r;
  cudaStream_t st = P->st;
  const int64_t Lg = std::max<int64_t>(1024, (q + 8 * ctx->num_sms - 1) / (8 * ctx->num_sms));
  if (!P->gseg) {
    const int64_t gnp = (int64_t)n + (q + Lg - 1) / Lg + 1;
    const size_t extra = (size_t)gnp * (3 * sizeof(int32_t) + rr * sizeof(double)) +
                         (size_t)n * (3 * sizeof(int32_t)) + 64 +
                         exclusive_scan_tmp_bytes(n);
    if (ctx->budget && ctx->in_use + extra > ctx->budget)
      return fail(ctx, CPHIFI_E_ADMISSION, "Gram blocks exceed the HBM budget");
    P->gnp = (int)gnp;
    int64_t* scan_tmp = nullptr;
    CK(dalloc(P, &P->gseg, (size_t)gnp));
    CK(dalloc(P, &P->gbeg, (size_t)gnp));
    CK(dalloc(P, &P->gend, (size_t)gnp));
    CK(dalloc(P, &P->gfirst, (size_t)n + 1));
    CK(dalloc(P, &P->gcount, (size_t)n));
    CK(dalloc(P, &P->gticket, (size_t)n));
    CK(dalloc(P, &P->gpart, (size_t)gnp * rr));
    CK(dalloc(P, &scan_tmp, exclusive_scan_tmp_bytes(n) / sizeof(int64_t) + 1));
    CK(cudaMemsetAsync(P->gticket, 0, (size_t)n * sizeof(unsigned), st));
    CK(launch_piece_counts(P->row_ptr, n, Lg, P->gcount, nullptr, st));
    CK(exclusive_scan_i32(P->gcount, P->gfirst, n, scan_tmp, exclusive_scan_tmp_bytes(n), st));
    CK(launch_piece_fill(P->row_ptr, n, Lg, P->gfirst, P->gcount, P->gseg, P->gbeg, P->gend,
                         nullptr, st));
  }
  const PieceList pl{P->gseg, P->gbeg, P->gend, P->gfirst, P->gcount, P->gticket, nullptr,
                     P->gnp, 0, nullptr};
  const int grid = std::max(1, std::min(P->gnp, ctx->num_sms * 8));
  if (want32 && !P->c32_ok) {
    if (ctx->budget && ctx->in_use + (size_t)n * rr * sizeof(float) > ctx->budget)
      return fail(ctx, CPHIFI_E_ADMISSION, "Gram blocks exceed the HBM budget");
    if (!P->C32) CK(dalloc(P, &P->C32, (size_t)n * rr));
    CK(launch_gram_build_f32(pl, P->gfirst + n, grid, P->zhi, r, (float*)P->gpart, P->C32, st));
    P->c32_ok = true;
  }
  if (want64 && !P->c64_ok) {
    if (ctx->budget && ctx->in_use + (size_t)n * rr * sizeof(double) > ctx->budget)
      return fail(ctx, CPHIFI_E_ADMISSION, "Gram blocks exceed the HBM budget");
    if (!P->C64) CK(dalloc(P, &P->C64, (size_t)n * rr));
    CK(launch_gram_build_df(pl, P->gfirst + n, grid, P->zhi, P->zhi ? nullptr : P->z64, r,
                            P->gpart, P->C64, st));
    P->c64_ok = true;
  }
  return CPHIFI_OK;
}

}  // namespace

// One PCG solve as a resumable sequence of device work (§4.4): begin() queues
// the right-hand side and the start; each advance() runs when the previous
// step's work (and its copy of the device scalars) has finished, decides from
// the scalars, and queues the next step.  The synchronous solve loops over it;
// submitted requests interleave the steps of many solves on their own
// streams.  Between steps the host reads a few scalars; nothing else.
struct SolveRun {
  enum Stage { INIT, CHUNK, CONFIRM, LASTRES, FINAL, DONE };
  cphifi_problem* P;
  cphifi_params prm;
  const double* W0;
  double* W_out;
  int mem;
  int prec;
  bool mixed, emul;
  cudaStream_t st;
  Timer tm;
  Launcher L;
  Stage stage = INIT;
  bool converged = false;
  int status = CPHIFI_OK;
  int64_t pass = 0;
  int tcerr = 0;
  std::chrono::steady_clock::time_point t0;
  // CUDA graphs of the iteration chunk (launch-bound small problems):
  // captured on first use per chunk length; profiling runs launch directly.
  bool use_graphs;
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;
  std::vector<int64_t> graph_launches;  // kernels captured in each graph
  double chunk_build_ms = 0.0;  // host time of building the chunk graphs

  SolveRun(cphifi_problem* p, const cphifi_params& pr, const double* w0, double* wout, int m,
           bool graphs_ok)
      : P(p), prm(pr), W0(w0), W_out(wout), mem(m), prec(pr.precision),
        mixed(is_lowp(pr.precision)), emul(pr.precision != CPHIFI_FP64), st(p->st),
        tm(p->st, pr.profile != 0), L{p, p->st, &tm},
        use_graphs(graphs_ok && pr.profile == 0) {
    L.gram = pr.gram;
  }
  ~SolveRun() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
  }
  SolveRun(const SolveRun&) = delete;
  SolveRun& operator=(const SolveRun&) = delete;

  cphifi_ctx* ctx() const { return P->ctx; }
  int* tc_word() const { return reinterpret_cast<int*>(P->hs + 1); }
  int* err_word() const { return reinterpret_cast<int*>(P->hs + 1) + 1; }
  int err(cudaError_t e, const char* what) {
    ctx()->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    status = CPHIFI_E_DEVICE;
    stage = DONE;
    return CPHIFI_E_DEVICE;
  }
#define SR_CK(...)                                   \
  do {                                               \
    cudaError_t e_ = (__VA_ARGS__);                  \
    if (e_ != cudaSuccess) return err(e_, #__VA_ARGS__); \
  } while (0)

  // Queue the copy of the device scalars and the event that marks the end of
  // the queued step.
  int mark() {
    SR_CK(cudaMemcpyAsync(P->hs, P->s, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    SR_CK(cudaEventRecord(P->ev[4], st));
    return CPHIFI_OK;
  }
  bool ready() const { return stage == DONE || cudaEventQuery(P->ev[4]) != cudaErrorNotReady; }
  int wait_ready() {
    if (stage == DONE) return CPHIFI_OK;
    SR_CK(cudaEventSynchronize(P->ev[4]));
    return CPHIFI_OK;
  }

  int begin() {
    t0 = std::chrono::steady_clock::now();
    const int n = P->n, r = P->r;
    const size_t nr = (size_t)n * r;
    DevScalars h{};
    h.tol2 = prm.tol * prm.tol;
    h.lam = prm.lambda;
    h.rho = prm.rho;
    h.max_iter = prm.max_iter;
    h.mode = mixed ? 1 : 0;
    SR_CK(cudaEventRecord(P->ev[0], st));
    if (prm.gram) {  // the Gram blocks this solve uses (built once per problem)
      const int rc = ensure_grams(P, mixed, !mixed || prm.gram == 2);
      if (rc != CPHIFI_OK) {
        status = rc;
        stage = DONE;
        return rc;
      }
    }
    SR_CK(cudaMemcpyAsync(P->s, &h, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
    if (P->tc_err) SR_CK(cudaMemsetAsync(P->tc_err, 0, sizeof(int), st));
    SR_CK(launch_build_D(P->kern->dK, P->dV, n, r, P->gamma, prm.lambda, prm.rho, P->D64, P->D32, st));
    // right-hand side in the eigenbasis: bbar = D_K U_K' B, and ||bbar||^2
    SR_CK(L.utb(emul, CM_DK_NORM, P->Bm, P->bbar, P->s));
    // start: x = U_K' W0 (or 0) and its true residual
    if (W0) {
      SR_CK(upload(P->tmp64, W0, nr * sizeof(double), mem, st));
      SR_CK(L.utb(emul, CM_STORE, P->tmp64, P->x, P->s));
      SR_CK(L.opwide(emul, CM_RESID, P->x, P->res, P->s, nullptr, 0));
    } else {
      SR_CK(cudaMemsetAsync(P->x, 0, nr * sizeof(double), st));
      SR_CK(cudaMemcpyAsync(P->res, P->bbar, nr * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    SR_CK(L.restart(prec));
    SR_CK(cudaEventRecord(P->ev[1], st));
    stage = INIT;
    *err_word() = 0;
    SR_CK(cudaMemcpyAsync(err_word(), P->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return mark();
  }

  // m PCG iterations (plus, in the mixed modes, the FP64-accurate true
  // residual and restart that close every cycle).
  int queue_chunk(int m) {
    if (!use_graphs) {
      for (int k = 0; k < m; ++k) SR_CK(L.iteration(prec));
      if (mixed) SR_CK(L.true_residual_check(prec));
      return CPHIFI_OK;
    }
    cudaGraphExec_t ex = nullptr;
    int64_t nl = 0;
    for (size_t k = 0; k < graphs.size(); ++k)
      if (graphs[k].first == m) { ex = graphs[k].second; nl = graph_launches[k]; }
    if (!ex) {
      const auto tb = std::chrono::steady_clock::now();
      cudaGraph_t g = nullptr;
      const int64_t before = L.launches;
      SR_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < m && e == cudaSuccess; ++k) e = L.iteration(prec);
      if (e == cudaSuccess && mixed) e = L.true_residual_check(prec);
      cudaError_t e2 = cudaStreamEndCapture(st, &g);
      nl = L.launches - before;
      L.launches = before;
      if (e != cudaSuccess) return err(e, "capturing the iteration chunk");
      SR_CK(e2);
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      SR_CK(e);
      graphs.push_back({m, ex});
      graph_launches.push_back(nl);
      chunk_build_ms += std::chrono::duration<double, std::milli>(
                            std::chrono::steady_clock::now() - tb).count();
    }
    SR_CK(cudaGraphLaunch(ex, st));
    L.launches += nl;
    return CPHIFI_OK;
  }

  int queue_final() {
    const size_t nr = (size_t)P->n * P->r;
    SR_CK(cudaEventRecord(P->ev[2], st));
    double* Wdev = (mem == CPHIFI_MEM_DEVICE) ? W_out : P->tmp64;
    SR_CK(L.ux(emul, P->x, Wdev, P->s));
    if (mem != CPHIFI_MEM_DEVICE) SR_CK(download(W_out, Wdev, nr * sizeof(double), mem, st));
    SR_CK(cudaEventRecord(P->ev[3], st));
    if (P->tc_err)
      SR_CK(cudaMemcpyAsync(tc_word(), P->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    stage = FINAL;
    return mark();
  }

  // The scalars of the finished step decide the next one.
  int advance() {
    const DevScalars* hs = P->hs;
    switch (stage) {
      case INIT:
        if (*err_word()) {  // input errors of an asynchronous creation
          status = CPHIFI_E_INVALID_ARG;
          ctx()->last_error = input_error_text(*err_word());
          stage = DONE;
          return CPHIFI_OK;
        }
        if (hs->bb == 0.0) {  // b = 0: W = 0 solves the system exactly
          converged = true;
          SR_CK(cudaMemsetAsync(P->x, 0, (size_t)P->n * P->r * sizeof(double), st));
          return queue_final();
        }
        if (W0 && hs->done) {  // the warm start already meets the tolerance
          converged = true;
          return queue_final();
        }
        stage = CHUNK;
        return next_chunk();
      case CHUNK:
        if (hs->status) return finish_loop();
        if (mixed) {
          if (hs->done) { converged = true; return finish_loop(); }
          // Restart from the true residual when the recurrence has stopped
          // (it met the tolerance, or max_iter) or has drifted below the true
          // residual by more than a factor 2: the low-precision operator's
          // error then dominates.  Otherwise PCG runs on with its Krylov
          // space intact.
          if (hs->inner_done || hs->rr < 0.25 * hs->true_rr) {
            if (prm.max_iter - hs->iter <= 0) return last_residual();
            SR_CK(L.adopt_restart(prec));
          }
          return next_chunk();
        }
        if (hs->done) {
          // FP64-accurate operator: the recurrence met tol; confirm with the
          // true residual and restart from it if it does not (refinement).
          SR_CK(L.true_residual_restart(prec));
          stage = CONFIRM;
          return mark();
        }
        return next_chunk();
      case CONFIRM:
        if (hs->status) return finish_loop();
        if (hs->done) { converged = true; return finish_loop(); }
        stage = CHUNK;
        return next_chunk();
      case LASTRES:
        if (hs->done) converged = true;
        return finish_loop();
      case FINAL: {
        tcerr = P->tc_err ? *tc_word() : 0;
        if (tcerr) {
          status = CPHIFI_E_TIMEOUT;  // a bounded wait in a tensor-core product expired
          ctx()->last_error = "tensor-core product: a bounded wait expired (error code " +
                              std::to_string(tcerr) + ")";
        }
        stage = DONE;
        return CPHIFI_OK;
      }
      case DONE:
        return CPHIFI_OK;
    }
    return CPHIFI_OK;
  }

  int next_chunk() {
    const DevScalars* hs = P->hs;
    const int cycle = mixed ? std::max(1, prm.k_replace) : std::max(1, prm.check_every);
    const int left = prm.max_iter - hs->iter;
    // Every chunk adds iterations or the loop ends; the pass bound is a second
    // guarantee that it terminates.
    if (left <= 0 || ++pass > (int64_t)prm.max_iter + 2) return last_residual();
    const int m = std::min(cycle, left);
    int rc = queue_chunk(m);
    if (rc != CPHIFI_OK) return rc;
    stage = CHUNK;
    return mark();
  }

  // max_iter reached: the true residual of the returned iterate.
  int last_residual() {
    if (P->hs->status) return finish_loop();
    SR_CK(L.opwide(emul, CM_RESID, P->x, P->res, P->s, nullptr, 0));
    stage = LASTRES;
    return mark();
  }

  int finish_loop() {
    const DevScalars* hs = P->hs;
    if (hs->status) status = hs->status;
    else if (!converged) status = CPHIFI_E_NOT_CONVERGED;
    return queue_final();
  }
#undef SR_CK

  void fill(cphifi_stats* stats) {
    auto t1 = std::chrono::steady_clock::now();
    const DevScalars* hs = P->hs;
    memset(stats, 0, sizeof(*stats));
    stats->status = status;
    stats->iterations = hs->iter;
    stats->true_residuals = hs->true_evals;
    stats->restarts = hs->restarts;
    const double bn = std::sqrt(hs->bb);
    stats->rel_residual = hs->bb > 0 ? std::sqrt(hs->true_rr) / bn : 0.0;
    if (hs->true_evals == 0) stats->rel_residual = hs->bb > 0 ? std::sqrt(hs->rr) / bn : 0.0;
    stats->rel_residual_recurrence = hs->bb > 0 ? std::sqrt(hs->rr) / bn : 0.0;
    stats->solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    stats->kernel_launches = L.launches;
    stats->graph_build_ms = chunk_build_ms;
    stats->setup_launches = P->create_launches;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P->ev[0], P->ev[1]) == cudaSuccess) stats->rhs_ms = ms;
    if (cudaEventElapsedTime(&ms, P->ev[1], P->ev[2]) == cudaSuccess) stats->iter_ms = ms;
    if (cudaEventElapsedTime(&ms, P->ev[2], P->ev[3]) == cudaSuccess) stats->final_ms = ms;
    if (tm.on) {
      stats->gds_ms = Timer::total(tm.gds);
      stats->gds_launches = (int)tm.gds.size();
      stats->gemm_ms = Timer::total(tm.gemm);
      stats->gemm_launches = (int)tm.gemm.size();
      stats->gds64_ms = Timer::total(tm.gds64);
      stats->gds64_launches = (int)tm.gds64.size();
      stats->gemm64_ms = Timer::total(tm.gemm64);
      stats->gemm64_launches = (int)tm.gemm64.size();
    }
  }
};

// Checks that do not touch the device, then the operator data the precision
// needs.
// ------------------------------------------------ alternating fit (§2) ----
// Rebuilds what depends on the finite factors (their double-float rows, V,
// eig(V), Zhat, the MTTKRP B) from the kept sorted observation lists; the
// order, pieces and density are unchanged.  Synchronous; input errors (a
// non-finite factor) give CPHIFI_E_INVALID_ARG.
static int problem_rebuild(cphifi_problem* P) {
  cphifi_ctx* ctx = P->ctx;
  cudaStream_t st = P->st;
  const int r = P->r, d = P->d_other;
  P->c32_ok = P->c64_ok = false;  // the Gram blocks follow Zhat
  CK(cudaMemsetAsync(P->err, 0, sizeof(int), st));
  for (int m = 0; m < d; ++m) {
    CK(launch_validate_dense(P->factors[m], P->sizes[m] * r, P->err, st));
    CK(launch_split_rows_df(P->factors[m], P->sizes[m], r, P->fhl[m], st));
  }
  CK(launch_gram(P->factors_dev, P->sizes_dev, d, r, P->V, st));
  CK(launch_jacobi_eig(P->V, r, P->dV, P->UV, 60, P->info, st));
  CK(launch_convert<double, float>(P->UV, P->UV32, (int64_t)r * r, st));
  // the same pass as the problem's creation, so a rebuilt problem gives the
  // bits of one created from the new factors
  std::vector<std::pair<void*, size_t>> tmps;
  auto alloc = [&](size_t bytes) -> void* {
    void* ptr = nullptr;
    size_t got = 0;
    if (pool_alloc(ctx, std::max<size_t>(bytes, 1), &ptr, &got) != cudaSuccess) return nullptr;
    tmps.push_back({ptr, got});
    return ptr;
  };
  const cudaError_t ez = zhat_and_rhs(P, nullptr, P->oidx_s, P->vals_s, nullptr, alloc, st);
  int herr = 0;
  cudaError_t ec = cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  const cudaError_t es = cudaStreamSynchronize(st);
  for (auto& t : tmps) pool_release(ctx, t.first, t.second);
  CK(ez);
  CK(ec);
  CK(es);
  if (herr) return fail(ctx, CPHIFI_E_INVALID_ARG, input_error_text(herr));
  P->stale = false;
  return CPHIFI_OK;
}

// A_k = K W = U_K (D_K o (U_K' W)) in FP64 into P->Ak; W is a device n x r
// array (column-major).
static cudaError_t kernel_factor(cphifi_problem* P, const double* Wd) {
  const cphifi_kernel* K = P->kern;
  if (K->pts) {  // K generated from the points, FP64; partials in cpart
    const int cap = std::max(std::max(P->nsplit64, P->nsplit32), std::max(P->nsplitdf, P->nsplittc));
    const int ns = std::min(kpoints_pick_split(P->n, P->ctx->num_sms), cap);
    return launch_kpoints_apply(true, K->pts, P->n, K->dim, K->kind, K->bandwidth, P->r, Wd,
                                P->Ak, ns, (double*)P->cpart, P->st);
  }
  Launcher L{P, P->st, nullptr};
  double* Cp = (double*)P->cpart;
  cudaError_t e = L.gemm64(false, nullptr, Wd, Cp, nullptr, 0);
  if (e == cudaSuccess) e = L.combine<double, double>(CM_STORE, Cp, nullptr, nullptr, P->tmp64b,
                                                      P->s2, nullptr, P->nsplit64);
  if (e == cudaSuccess) e = L.gemm64(true, P->kern->dK, P->tmp64b, Cp, nullptr, 0);
  if (e == cudaSuccess) e = L.combine<double, double>(CM_STORE, Cp, nullptr, nullptr, P->Ak, P->s2,
                                                      nullptr, P->nsplit64);
  return e;
}

// W (host or device) into P->tmp64, then A_k.
static int load_weights(cphifi_problem* P, const double* W, int mem) {
  cphifi_ctx* ctx = P->ctx;
  if (!W) return fail(ctx, CPHIFI_E_INVALID_ARG, "null W");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  CK(upload(P->tmp64, W, (size_t)P->n * P->r * sizeof(double), mem, P->st));
  CK(launch_validate_dense(P->tmp64, (int64_t)P->n * P->r, P->err, P->st));
  CK(kernel_factor(P, P->tmp64));
  return CPHIFI_OK;
}

static int update_factor(cphifi_problem* P, int m, const double* W, double* A_out, int mem) {
  cphifi_ctx* ctx = P->ctx;
  if (!P->keep_obs) return fail(ctx, CPHIFI_E_INVALID_ARG, "problem created without CPHIFI_KEEP_OBS");
  if (m < 0 || m >= P->d_other) return fail(ctx, CPHIFI_E_INVALID_ARG, "mode out of range");
  cudaStream_t st = P->st;
  const int64_t q = P->q;
  const int64_t nm = P->sizes[m];
  if (nm > (int64_t(1) << 30)) return fail(ctx, CPHIFI_E_UNSUPPORTED, "finite mode too large");
  CK(cudaMemsetAsync(P->err, 0, sizeof(int), st));
  if (!P->perm_m[m]) {  // the mode-m order of the observations, once
    CK(dalloc(P, &P->perm_m[m], (size_t)std::max<int64_t>(q, 1)));
    CK(dalloc(P, &P->rowp_m[m], (size_t)nm + 1));
    void* keys = nullptr;
    void* rtmp = nullptr;
    size_t gk = 0, gr = 0;
    CK(pool_alloc(ctx, (size_t)std::max<int64_t>(q, 1) * sizeof(uint32_t), &keys, &gk));
    cudaError_t e = pool_alloc(ctx, radix_sort_tmp_bytes(q), &rtmp, &gr);
    if (e == cudaSuccess) e = launch_mode_keys(q, P->d_other, m, P->oidx_s, (uint32_t*)keys, st);
    if (e == cudaSuccess) e = launch_iota(P->perm_m[m], q, st);
    if (e == cudaSuccess && q > 1)
      e = radix_sort_pairs((uint32_t*)keys, P->perm_m[m], q, bits_for((int)nm), rtmp, st);
    if (e == cudaSuccess) e = launch_row_ptr((const uint32_t*)keys, q, (int)nm, P->rowp_m[m], st);
    cudaStreamSynchronize(st);
    if (rtmp) pool_release(ctx, rtmp, gr);
    pool_release(ctx, keys, gk);
    CK(e);
  }
  int rc = load_weights(P, W, mem);
  if (rc != CPHIFI_OK) return rc;
  CK(cudaMemsetAsync(P->nfail, 0, sizeof(int), st));
  CK(launch_als_rows((int)nm, m, P->d_other, P->r, P->n, P->rowp_m[m], P->perm_m[m], P->kidx_s,
                     P->oidx_s, P->vals_s, P->Ak, (const double* const*)P->factors_dev,
                     P->sizes_dev, P->factors[m], P->nfail, ctx->num_sms, st));
  if (A_out) CK(download(A_out, P->factors[m], (size_t)nm * P->r * sizeof(double), mem, st));
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  P->stale = true;
  if (herr) return fail(ctx, CPHIFI_E_INVALID_ARG, "non-finite weight W");
  return CPHIFI_OK;
}

static int problem_fit(cphifi_problem* P, const double* W, int mem, double* res2, double* t2) {
  cphifi_ctx* ctx = P->ctx;
  if (!P->keep_obs) return fail(ctx, CPHIFI_E_INVALID_ARG, "problem created without CPHIFI_KEEP_OBS");
  cudaStream_t st = P->st;
  CK(cudaMemsetAsync(P->err, 0, sizeof(int), st));
  int rc = load_weights(P, W, mem);
  if (rc != CPHIFI_OK) return rc;
  double h[2] = {0.0, 0.0};
  if (P->q > 0) {
    CK(launch_fit(P->q, P->d_other, P->r, P->n, P->kidx_s, P->oidx_s, P->vals_s, P->Ak,
                  (const double* const*)P->factors_dev, P->sizes_dev, P->red, P->fit2,
                  ctx->num_sms, st));
    CK(cudaMemcpyAsync(h, P->fit2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (herr) return fail(ctx, CPHIFI_E_INVALID_ARG, "non-finite weight W");
  if (res2) *res2 = h[0];
  if (t2) *t2 = h[1];
  return CPHIFI_OK;
}

static int solve_prepare(cphifi_problem* P, const cphifi_params* prm, double* W_out, int mem) {
  cphifi_ctx* ctx = P->ctx;
  int rc = check_params(ctx, prm);
  if (rc != CPHIFI_OK) return rc;
  if (!W_out) return fail(ctx, CPHIFI_E_INVALID_ARG, "null W_out");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  if (P->stale) {
    const int rc = problem_rebuild(P);
    if (rc != CPHIFI_OK) return rc;
  }
  const int prec = prm->precision;
  if (is_tc(prec) && !P->kern->tc)
    return fail(ctx, CPHIFI_E_UNSUPPORTED, "tensor-core products unavailable for this kernel");
  if (prec == CPHIFI_MIXED_BF16X3 && !P->ozb)
    return fail(ctx, CPHIFI_E_UNSUPPORTED, "BF16 slices of U_K unavailable for this kernel");
  return prec != CPHIFI_FP64 ? ensure_lowp(P) : ensure_fp64(P);
}

extern "C" int cphifi_problem_solve(cphifi_problem* P, const cphifi_params* prm, const double* W0,
                                    double* W_out, int mem, cphifi_stats* stats) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  Enter guard(ctx);
  int rc = solve_prepare(P, prm, W_out, mem);
  if (rc != CPHIFI_OK) return rc;
  SolveRun run(P, *prm, W0, W_out, mem, /*graphs_ok=*/false);
  rc = run.begin();
  while (rc == CPHIFI_OK && run.stage != SolveRun::DONE) {
    if ((rc = run.wait_ready()) != CPHIFI_OK) break;
    rc = run.advance();
  }
  if (rc != CPHIFI_OK) return rc;
  if (stats) run.fill(stats);
  if (run.status != CPHIFI_OK && run.status != CPHIFI_E_TIMEOUT)
    ctx->last_error = std::string("solve: ") + cphifi_status_string(run.status);
  return run.status;
}

extern "C" int cphifi_solve(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                            const int64_t* other_sizes, const double* const* factors, int32_t r,
                            int64_t q, const int32_t* kidx, const int32_t* oidx,
                            const void* vals, uint32_t flags, const cphifi_params* params,
                            const double* W0, double* W_out, int mem, cphifi_stats* stats) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  int rc = check_params(ctx, params);
  if (rc != CPHIFI_OK) return rc;
  flags |= params->precision == CPHIFI_FP64 ? CPHIFI_NEED_FP64 : CPHIFI_NEED_LOWP;
  auto t0 = std::chrono::steady_clock::now();
  cphifi_problem* P = nullptr;
  rc = cphifi_problem_create(ctx, kern, d_other, other_sizes, factors, r, q, kidx, oidx, vals,
                             flags, mem, &P);
  if (rc != CPHIFI_OK) return rc;
  auto t1 = std::chrono::steady_clock::now();
  rc = cphifi_problem_solve(P, params, W0, W_out, mem, stats);
  if (stats) stats->setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  std::string keep = ctx->last_error;
  cphifi_problem_destroy(P);
  ctx->last_error = keep;
  return rc;
}

// ------------------------------------------------ submitted requests -----
// Admission classes: a request whose device footprint exceeds
// kLargeRequestBytes is large; large requests hold at most a quarter of the
// slots (at least one).  A pending request older than kAdmitAgeMs is no
// longer overtaken by newer ones.
constexpr size_t kLargeRequestBytes = size_t(1) << 30;
constexpr double kAdmitAgeMs = 50.0;

struct Request {
  uint64_t id = 0;
  const cphifi_kernel* kern = nullptr;
  int32_t d_other = 0;
  std::vector<int64_t> sizes;
  std::vector<const double*> factors;
  int32_t r = 0;
  int64_t q = 0;
  const int32_t* kidx = nullptr;
  const int32_t* oidx = nullptr;
  const void* vals = nullptr;
  uint32_t flags = 0;
  cphifi_params prm{};
  const double* W0 = nullptr;
  double* W_out = nullptr;
  int mem = 0;
  size_t need = 0;
  bool large = false;  // footprint above kLargeRequestBytes (admission class)
  enum { PENDING, ACTIVE, DONE } state = PENDING;
  cphifi_problem* P = nullptr;
  std::unique_ptr<SolveRun> run;
  cudaEvent_t ev_submit = nullptr;  // inputs ready (caller's stream order)
  int slot = -1;
  int status = CPHIFI_OK;
  std::string error;
  cphifi_stats stats{};
  std::chrono::steady_clock::time_point t_submit, t_admit, t_created;
};

namespace {

void request_finish(cphifi_ctx* ctx, Request* R, int status) {
  if (R->run) {
    if (status == CPHIFI_OK && R->run->stage == SolveRun::DONE) {
      R->run->fill(&R->stats);
      status = R->run->status;
    }
    R->run.reset();
  }
  R->stats.status = status;
  R->stats.queue_ms =
      std::chrono::duration<double, std::milli>(R->t_admit - R->t_submit).count();
  R->stats.setup_ms =
      std::chrono::duration<double, std::milli>(R->t_created - R->t_admit).count();
  if (status != CPHIFI_OK && R->error.empty()) R->error = ctx->last_error;
  if (R->P) {
    cphifi_problem_destroy(R->P);
    R->P = nullptr;
  }
  if (R->slot >= 0) {
    ctx->slot_busy[R->slot] = false;
    R->slot = -1;
  }
  if (R->ev_submit) {
    cudaEventDestroy(R->ev_submit);
    R->ev_submit = nullptr;
  }
  R->status = status;
  R->state = Request::DONE;
  ctx->done_unreported.push_back(R->id);
}

// Advance every active request whose queued step has finished; admit
// pending requests while a slot and the HBM budget allow.  Returns whether
// anything changed.
bool progress(cphifi_ctx* ctx) {
  bool moved = false;
  deferred_collect(ctx, false);
  for (size_t k = 0; k < ctx->active.size();) {
    Request* R = ctx->active[k];
    int rc = CPHIFI_OK;
    if (R->run->ready()) {
      moved = true;
      rc = R->run->advance();
    }
    if (rc != CPHIFI_OK || R->run->stage == SolveRun::DONE) {
      request_finish(ctx, R, rc);
      ctx->active.erase(ctx->active.begin() + k);
      moved = true;
    } else {
      ++k;
    }
  }
  // Size-aware admission: pending requests are considered oldest first, and
  // one that cannot start yet (its footprint does not fit the budget next to
  // the running ones, or it is large and the slots large requests may hold
  // are taken) is passed over by the smaller ones behind it, so that a large
  // request waiting for memory does not hold up the small ones.  A request
  // that has waited longer than kAdmitAgeMs is passed over by nobody: from it
  // on, admission is in submission order until it starts.
  const auto now = std::chrono::steady_clock::now();
  int large_active = 0;
  for (const Request* A : ctx->active) large_active += A->large ? 1 : 0;
  const int max_large = std::max(1, ctx->max_active / 4);
  size_t cand = 0;
  while (cand < ctx->pending.size() && (int)ctx->active.size() < ctx->max_active) {
    Request* R = ctx->pending[cand];
    deferred_collect(ctx, false);
    const bool aged =
        std::chrono::duration<double, std::milli>(now - R->t_submit).count() > kAdmitAgeMs;
    if (ctx->budget && ctx->in_use + ctx->deferred_bytes + R->need > ctx->budget) {
      if (ctx->active.empty() && !ctx->deferred.empty()) {
        deferred_collect(ctx, true);  // empties the list: runs once per request
        continue;
      }
      if (ctx->active.empty()) {  // cannot fit even alone
        ctx->pending.erase(ctx->pending.begin() + cand);
        R->error = "request footprint exceeds the HBM budget";
        request_finish(ctx, R, CPHIFI_E_ADMISSION);
        moved = true;
        continue;
      }
      if (aged) break;  // wait for memory to free up; nothing newer goes first
      ++cand;
      continue;
    }
    if (R->large && large_active >= max_large) {
      if (aged) break;
      ++cand;
      continue;
    }
    int slot = -1;
    for (int k = 0; k < (int)ctx->slot_busy.size(); ++k)
      if (!ctx->slot_busy[k]) { slot = k; break; }
    if (slot < 0) {
      cudaStream_t stn = nullptr;
      if (cudaStreamCreateWithFlags(&stn, cudaStreamNonBlocking) != cudaSuccess) break;
      ctx->slot_stream.push_back(stn);
      ctx->slot_busy.push_back(false);
      slot = (int)ctx->slot_stream.size() - 1;
    }
    ctx->pending.erase(ctx->pending.begin() + cand);
    large_active += R->large ? 1 : 0;
    moved = true;
    R->t_admit = std::chrono::steady_clock::now();
    ctx->slot_busy[slot] = true;
    R->slot = slot;
    int rc = cudaStreamWaitEvent(ctx->slot_stream[slot], R->ev_submit, 0) == cudaSuccess
                 ? (int)CPHIFI_OK
                 : fail(ctx, CPHIFI_E_DEVICE, "ordering the request after its inputs");
    if (rc == CPHIFI_OK)
      rc = problem_create_on(ctx, R->kern, R->d_other, R->sizes.data(), R->factors.data(), R->r,
                               R->q, R->kidx, R->oidx, R->vals, R->flags, R->mem,
                               ctx->slot_stream[slot], /*async=*/true, &R->P);
    R->t_created = std::chrono::steady_clock::now();
    if (rc == CPHIFI_OK) rc = solve_prepare(R->P, &R->prm, R->W_out, R->mem);
    if (rc == CPHIFI_OK) {
      R->run.reset(new SolveRun(R->P, R->prm, R->W0, R->W_out, R->mem, /*graphs_ok=*/true));
      rc = R->run->begin();
    }
    if (rc != CPHIFI_OK) {
      request_finish(ctx, R, rc);
      continue;
    }
    R->state = Request::ACTIVE;
    ctx->active.push_back(R);
  }
  return moved;
}

}  // namespace

static bool kernel_in_use(const cphifi_ctx* ctx, const cphifi_kernel* kern) {
  for (const auto& kv : ctx->requests)
    if (kv.second->kern == kern && kv.second->state != Request::DONE) return true;
  return false;
}

static void requests_clear(cphifi_ctx* ctx) {
  for (auto& kv : ctx->requests) {
    Request* R = kv.second;
    if (R->P) cudaStreamSynchronize(R->P->st);
    if (R->state != Request::DONE) request_finish(ctx, R, CPHIFI_E_INVALID_ARG);
    delete R;
  }
  ctx->requests.clear();
  ctx->pending.clear();
  ctx->active.clear();
  ctx->done_unreported.clear();
  for (auto stn : ctx->slot_stream) cudaStreamDestroy(stn);
  ctx->slot_stream.clear();
  ctx->slot_busy.clear();
}

extern "C" int cphifi_ctx_set_tuning(cphifi_ctx* ctx, int32_t n_log2, int32_t q_log2, int32_t r,
                                     const cphifi_tuning* t) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  if (n_log2 < 0 || n_log2 > 30 || q_log2 < 0 || q_log2 > 31 || r < 1 || r > kMaxRank)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "tuning bucket out of range");
  const auto key = std::make_tuple((int)n_log2, (int)q_log2, (int)r);
  if (!t) {
    ctx->tuning.erase(key);
    return CPHIFI_OK;
  }
  for (int v : {t->gds_warps_per_sm, t->split32, t->split_tc, t->split_wide, t->split64})
    if (v < 0 || v > 64) return fail(ctx, CPHIFI_E_INVALID_ARG, "tuning value out of [0, 64]");
  ctx->tuning[key] = *t;
  return CPHIFI_OK;
}

extern "C" int cphifi_ctx_set_slots(cphifi_ctx* ctx, int max_active) {
  if (!ctx || max_active < 1 || max_active > 1024) return CPHIFI_E_INVALID_ARG;
  ctx->max_active = max_active;
  return CPHIFI_OK;
}

extern "C" int cphifi_submit(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                             const int64_t* other_sizes, const double* const* factors, int32_t r,
                             int64_t q, const int32_t* kidx, const int32_t* oidx,
                             const void* vals, uint32_t flags, const cphifi_params* params,
                             const double* W0, double* W_out, int mem, cphifi_ticket* ticket) {
  if (!ctx || !ticket) return CPHIFI_E_INVALID_ARG;
  *ticket = 0;
  int rc = check_params(ctx, params);
  if (rc != CPHIFI_OK) return rc;
  if (!kern || kern->ctx != ctx) return fail(ctx, CPHIFI_E_INVALID_ARG, "kernel of another context");
  if (d_other < 1 || d_other > 16 || !other_sizes || !factors)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "bad other modes");
  if (r < 1 || r > kMaxRank || q < 0 || q >= (int64_t(1) << 31))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "r or q out of range");
  if (!W_out) return fail(ctx, CPHIFI_E_INVALID_ARG, "null W_out");
  if (q > 0 && (!kidx || !oidx || !vals)) return fail(ctx, CPHIFI_E_INVALID_ARG, "null observation list");
  for (int m = 0; m < d_other; ++m)
    if (other_sizes[m] < 1 || other_sizes[m] > (int64_t(1) << 31) - 1 || !factors[m])
      return fail(ctx, CPHIFI_E_INVALID_ARG, "bad other-mode size or null factor");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  Enter guard(ctx);
  Request* R = new Request();
  R->id = ctx->next_ticket++;
  R->kern = kern;
  R->d_other = d_other;
  R->sizes.assign(other_sizes, other_sizes + d_other);
  R->factors.assign(factors, factors + d_other);
  R->r = r;
  R->q = q;
  R->kidx = kidx;
  R->oidx = oidx;
  R->vals = vals;
  R->flags = flags | (params->precision == CPHIFI_FP64 ? CPHIFI_NEED_FP64 : CPHIFI_NEED_LOWP);
  R->prm = *params;
  R->W0 = W0;
  R->W_out = W_out;
  R->mem = mem;
  R->t_submit = R->t_admit = R->t_created = std::chrono::steady_clock::now();
  {
    size_t need = 0, tmp = 0;
    problem_need(ctx, kern, d_other, R->sizes, r, q, R->flags, &need, &tmp);
    R->need = need + tmp;
    R->large = R->need > kLargeRequestBytes;
  }
  if (cudaEventCreateWithFlags(&R->ev_submit, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(R->ev_submit, ctx->stream) != cudaSuccess) {
    if (R->ev_submit) cudaEventDestroy(R->ev_submit);
    delete R;
    return fail(ctx, CPHIFI_E_DEVICE, "recording the submit event");
  }
  ctx->requests[R->id] = R;
  ctx->pending.push_back(R);
  *ticket = R->id;
  progress(ctx);
  return CPHIFI_OK;
}

extern "C" int cphifi_poll(cphifi_ctx* ctx, int32_t* n_active, int32_t* n_pending,
                           cphifi_ticket* done, int32_t done_cap, int32_t* n_done) {
  if (!ctx || done_cap < 0 || (done_cap > 0 && !done)) return CPHIFI_E_INVALID_ARG;
  Enter guard(ctx);
  progress(ctx);
  if (n_active) *n_active = (int32_t)ctx->active.size();
  if (n_pending) *n_pending = (int32_t)ctx->pending.size();
  // Tickets that completed since they were last listed, oldest first.
  auto& du = ctx->done_unreported;
  size_t k = 0, m = 0;
  for (; k < du.size() && (int32_t)m < done_cap; ++k) {
    if (ctx->requests.count(du[k])) done[m++] = du[k];
  }
  du.erase(du.begin(), du.begin() + k);
  if (n_done) *n_done = (int32_t)m;
  return CPHIFI_OK;
}

extern "C" int cphifi_wait(cphifi_ctx* ctx, cphifi_ticket ticket, int64_t timeout_us,
                           cphifi_stats* stats) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  auto it = ctx->requests.find(ticket);
  if (it == ctx->requests.end()) return fail(ctx, CPHIFI_E_INVALID_ARG, "unknown ticket");
  Request* R = it->second;
  Enter guard(ctx);
  const auto t0 = std::chrono::steady_clock::now();
  while (R->state != Request::DONE) {
    const bool moved = progress(ctx);
    if (R->state == Request::DONE) break;
    if (timeout_us >= 0) {
      const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                          std::chrono::steady_clock::now() - t0).count();
      if (us >= timeout_us) return fail(ctx, CPHIFI_E_TIMEOUT, "request still running");
    }
    if (!moved) std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
  if (stats) *stats = R->stats;
  const int status = R->status;
  auto& du = ctx->done_unreported;
  du.erase(std::remove(du.begin(), du.end(), ticket), du.end());
  if (status != CPHIFI_OK) ctx->last_error = R->error;
  ctx->requests.erase(it);
  delete R;
  return status;
}

// ------------------------------------------- one persistent launch -------
// cphifi_solve_batch: every problem created without host waits on the
// context's batch streams, then one launch of the persistent kernel
// (batch.cu) over all solves.  The descriptors are ordered by the work of one
// PCG iteration (2 n^2 r for the two products, 2 q r for the gather-dot/
// scatter), smallest first: idle blocks serve the first request with a free
// tile, so the short phases of small requests (whose chains are as long as
// the large ones' and often longer) never queue behind the many tiles of a
// large request, and the large requests take the blocks left over.
constexpr int kBatchStreams = 16;

extern "C" int cphifi_ctx_set_batch_wait(cphifi_ctx* ctx, int32_t ms) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  if (ms < 1 || ms > 600000)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "batch wait not in [1, 600000] ms");
  ctx->batch_wait_ns = 1000000ll * ms;
  return CPHIFI_OK;
}

// k-range splits of a batch request's products: chunks of about 64 (FP32)
// and 32 (double-float) columns of U_K (a few k slabs per tile: the tiles
// are bound by the latency of their loads, and short ones run side by
// side), at most 64 splits, or the tuning table's splits.
static void batch_splits(const cphifi_ctx* ctx, int n, int64_t q, int r, BatchReq* d) {
  cphifi_tuning t{};
  auto it = ctx->tuning.find(std::make_tuple(floor_log2(n), floor_log2(std::max<int64_t>(q, 1)), r));
  if (it != ctx->tuning.end()) t = it->second;
  auto chunk = [n](int tuned, int target, int cap, int align) {
    int s = tuned > 0 ? tuned : (n + target - 1) / target;
    s = std::max(1, std::min(s, cap));
    int kc = (n + s - 1) / s;
    kc = (kc + align - 1) / align * align;
    return kc;
  };
  d->kc32 = chunk(t.split32, 64, 32, 16);
  d->s32 = (n + d->kc32 - 1) / d->kc32;
  d->kcdf = chunk(t.split_wide, 32, 32, 16);
  d->sdf = (n + d->kcdf - 1) / d->kcdf;
}

extern "C" int cphifi_solve_batch(cphifi_ctx* ctx, int32_t count, const cphifi_batch_item* items,
                                  const cphifi_params* prm, int mem, cphifi_stats* stats,
                                  cphifi_batch_info* info) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  if (count < 0 || count > 65535 || (count > 0 && !items))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "batch: count not in [0, 65535] or null items");
  int rc = check_params(ctx, prm);
  if (rc != CPHIFI_OK) return rc;
  if (prm->precision != CPHIFI_MIXED_FP32)
    return fail(ctx, CPHIFI_E_UNSUPPORTED, "batch: the persistent launch runs mixed FP32 solves");
  if (prm->gram != 0)
    return fail(ctx, CPHIFI_E_UNSUPPORTED, "batch: the persistent launch streams Zhat (gram 0)");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  if (info) memset(info, 0, sizeof(*info));
  if (count == 0) return CPHIFI_OK;
  for (int k = 0; k < count; ++k)
    if (!items[k].W_out)
      return fail(ctx, CPHIFI_E_INVALID_ARG, "batch item " + std::to_string(k) + ": null W_out");
  Enter guard(ctx);
  const auto t0 = std::chrono::steady_clock::now();
  while ((int)ctx->batch_streams.size() < std::min(count, kBatchStreams)) {
    cudaStream_t bs = nullptr;
    CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    ctx->batch_streams.push_back(bs);
  }
  for (auto& e : ctx->batch_ev)
    if (!e) CK(cudaEventCreate(&e));
  const int nstreams = (int)ctx->batch_streams.size();
  std::vector<cphifi_problem*> P(count, nullptr);
  void* ws = nullptr;
  size_t ws_bytes = 0;
  auto cleanup = [&]() {
    for (auto* p : P)
      if (p) cphifi_problem_destroy(p);
    if (ws) {
      cudaStreamSynchronize(ctx->stream);
      pool_release(ctx, ws, ws_bytes);
      ctx->in_use -= ws_bytes;
    }
  };
  // 1. the problems, on the batch streams, in order after the caller's work
  CK(cudaEventRecord(ctx->ev_in, ctx->stream));
  for (auto bs : ctx->batch_streams) CK(cudaStreamWaitEvent(bs, ctx->ev_in, 0));
  for (int k = 0; k < count; ++k) {
    const cphifi_batch_item& it = items[k];
    rc = problem_create_on(ctx, it.kern, it.d_other, it.other_sizes, it.factors, it.r, it.q,
                           it.kidx, it.oidx, it.vals, it.flags | CPHIFI_NEED_LOWP, mem,
                           ctx->batch_streams[k % nstreams], /*async=*/true, &P[k]);
    if (rc == CPHIFI_OK) rc = solve_prepare(P[k], prm, it.W_out, mem);
    if (rc != CPHIFI_OK) {
      const std::string why = ctx->last_error;
      cleanup();
      return fail(ctx, rc, "batch item " + std::to_string(k) + ": " + why);
    }
  }
  const double create_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  // 2. descriptors in descending order of one iteration's work
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  auto work = [&](int k) {
    const double n = P[k]->n, r = P[k]->r;
    return 2.0 * n * n * r + 2.0 * (double)P[k]->q * r;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) < work(b); });
  std::vector<BatchReq> reqs(count);
  std::vector<size_t> cp_off(count), red_off(count), p2_off(count);
  size_t bytes = 0;
  auto take = [&bytes](size_t b) {
    const size_t o = bytes;
    bytes += (b + 255) / 256 * 256;
    return o;
  };
  const size_t off_reqs = take(sizeof(BatchReq) * count);
  const size_t off_state = take(sizeof(BatchState) * count);
  const size_t off_scal = take(sizeof(DevScalars) * count);
  const size_t off_ctl = take(sizeof(BatchCtl));
  for (int j = 0; j < count; ++j) {
    cphifi_problem* p = P[order[j]];
    BatchReq& d = reqs[j];
    d.n = p->n;
    d.r = p->r;
    batch_splits(ctx, p->n, p->q, p->r, &d);
    const size_t nr = (size_t)p->n * p->r;
    cp_off[j] = take(std::max((size_t)d.s32 * sizeof(float), (size_t)d.sdf * sizeof(double)) * nr);
    p2_off[j] = take(sizeof(double) * nr);
    red_off[j] = take(2 * sizeof(double) * (size_t)((p->n + kBatchRows - 1) / kBatchRows));
  }
  {
    size_t got = 0;
    CK(pool_alloc(ctx, bytes, &ws, &got));
    ws_bytes = got;
    ctx->in_use += got;
  }
  char* wb = static_cast<char*>(ws);
  std::vector<BatchState> st0(count);
  std::vector<DevScalars> sc0(count);
  for (int j = 0; j < count; ++j) {
    const int k = order[j];
    cphifi_problem* p = P[k];
    BatchReq& d = reqs[j];
    d.max_iter = prm->max_iter;
    d.k_replace = std::max(1, prm->k_replace);
    d.tol2 = prm->tol * prm->tol;
    d.lam = prm->lambda;
    d.rho = prm->rho;
    d.gamma = p->gamma;
    d.UKhi = p->kern->UK32;
    d.UKlo = p->kern->UKlo;
    d.dK = p->kern->dK;
    d.dV = p->dV;
    d.UV32 = p->UV32;
    d.pl = PieceList{p->pseg, p->pbeg, p->pend, p->seg_first, p->seg_count, p->seg_ticket,
                     p->warp_first, p->npieces, p->nwarps, nullptr};
    d.zhi = p->zhi;
    d.Bm = p->Bm;
    d.err = p->err;
    d.x = p->x;
    d.res = p->res;
    d.p[0] = p->p;
    d.p[1] = reinterpret_cast<double*>(wb + p2_off[j]);
    d.z = p->z;
    d.y = p->y;
    d.bbar = p->bbar;
    d.tres = p->tres;
    d.D64 = p->D64;
    d.y164 = p->y164;
    d.D32 = p->D32;
    d.y132 = p->y132;
    d.cp32 = reinterpret_cast<float*>(wb + cp_off[j]);  // the FP32 and double-float
    d.cpd = reinterpret_cast<double*>(wb + cp_off[j]);  // partials are never live together
    d.gds_partial = p->gds_partial;
    d.red = reinterpret_cast<double*>(wb + red_off[j]);
    d.s = reinterpret_cast<DevScalars*>(wb + off_scal) + j;
    d.W = mem == CPHIFI_MEM_DEVICE ? items[k].W_out : p->tmp64;
    // a held item: zero tiles in its first phase, so no block ever claims it
    st0[j].claim = items[k].hold ? 0ull : batch_first_claim(d);
    DevScalars& h = sc0[j];
    memset(&h, 0, sizeof(h));
    h.tol2 = d.tol2;
    h.lam = d.lam;
    h.rho = d.rho;
    h.max_iter = d.max_iter;
    h.mode = 1;
  }
  BatchCtl ctl0{};
  // 3. inputs of the launch, after every creation; the launch
  for (int k = 0; k < nstreams; ++k) {
    cudaEvent_t e = nullptr;
    CK(event_get(ctx, &e));
    CK(cudaEventRecord(e, ctx->batch_streams[k]));
    CK(cudaStreamWaitEvent(ctx->stream, e, 0));
    ctx->events_free.push_back(e);
  }
  CK(cudaMemcpyAsync(wb + off_reqs, reqs.data(), sizeof(BatchReq) * count,
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(wb + off_state, st0.data(), sizeof(BatchState) * count,
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(wb + off_scal, sc0.data(), sizeof(DevScalars) * count,
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(wb + off_ctl, &ctl0, sizeof(BatchCtl), cudaMemcpyHostToDevice, ctx->stream));
  const int blocks = batch_blocks(ctx->num_sms);
  if (blocks < 1) {
    cleanup();
    return fail(ctx, CPHIFI_E_DEVICE, "batch: the persistent kernel does not fit an SM");
  }
  CK(cudaEventRecord(ctx->batch_ev[0], ctx->stream));
  CK(launch_batch(reinterpret_cast<const BatchReq*>(wb + off_reqs),
                  reinterpret_cast<BatchState*>(wb + off_state),
                  reinterpret_cast<const DevScalars*>(wb + off_scal),
                  reinterpret_cast<BatchCtl*>(wb + off_ctl), count, ctx->batch_wait_ns, blocks,
                  ctx->stream));
  CK(cudaEventRecord(ctx->batch_ev[1], ctx->stream));
  // 4. results: W (host memory: from each problem's staging array), scalars
  if (mem != CPHIFI_MEM_DEVICE)
    for (int j = 0; j < count; ++j) {
      const int k = order[j];
      CK(download(items[k].W_out, reqs[j].W, (size_t)reqs[j].n * reqs[j].r * sizeof(double), mem,
                  ctx->stream));
    }
  std::vector<DevScalars> sc(count);
  std::vector<BatchState> stf(count);
  BatchCtl ctl{};
  CK(cudaMemcpyAsync(sc.data(), wb + off_scal, sizeof(DevScalars) * count, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(stf.data(), wb + off_state, sizeof(BatchState) * count,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctl, wb + off_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  float kms = 0.f;
  cudaEventElapsedTime(&kms, ctx->batch_ev[0], ctx->batch_ev[1]);
  // 5. statuses and statistics, in the caller's order
  int first_bad = CPHIFI_OK;
  std::string bad_msg;
  for (int j = 0; j < count; ++j) {
    const int k = order[j];
    const DevScalars& h = sc[j];
    int status = CPHIFI_OK;
    if (stf[j].fail) status = CPHIFI_E_INVALID_ARG;
    else if (stf[j].phase != kBatchPhaseDone) status = CPHIFI_E_TIMEOUT;
    else if (h.status) status = h.status;
    else if (!h.done) status = CPHIFI_E_NOT_CONVERGED;
    if (stats) {
      cphifi_stats& o = stats[k];
      memset(&o, 0, sizeof(o));
      o.status = status;
      o.iterations = h.iter;
      o.true_residuals = h.true_evals;
      o.restarts = h.restarts;
      const double bn = std::sqrt(h.bb);
      o.rel_residual = h.bb > 0 ? std::sqrt(h.true_evals ? h.true_rr : h.rr) / bn : 0.0;
      o.rel_residual_recurrence = h.bb > 0 ? std::sqrt(h.rr) / bn : 0.0;
      o.setup_ms = create_ms;
      o.solve_ms = kms;
      o.iter_ms = stf[j].t_done > 0 && ctl.t_start > 0 ? 1e-6 * (double)(stf[j].t_done - ctl.t_start)
                                                       : kms;
      o.kernel_launches = 1;
      o.setup_launches = P[k]->create_launches;
    }
    if (status != CPHIFI_OK && first_bad == CPHIFI_OK) {
      first_bad = status;
      bad_msg = "batch item " + std::to_string(k) + ": " +
                (status == CPHIFI_E_INVALID_ARG ? std::string("invalid observations or factors")
                                                : std::string(cphifi_status_string(status)));
    }
  }
  if (info) {
    info->create_ms = create_ms;
    info->kernel_ms = kms;
    info->tiles = ctl.progress;
    info->blocks = blocks;
    info->timed_out = ctl.err;
  }
  cleanup();
  if (info)
    info->total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (first_bad != CPHIFI_OK) ctx->last_error = bad_msg;
  return first_bad;
}

// ------------------------------------------------- step-by-step calls -----
extern "C" int cphifi_problem_rhs(cphifi_problem* P, double* B_out, double* b_out, int mem) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  Enter guard(ctx);
  cudaStream_t st = P->st;
  const size_t nr = (size_t)P->n * P->r;
  Launcher L{P, st, nullptr};
  if (B_out) CK(download(B_out, P->Bm, nr * sizeof(double), mem, st));
  if (b_out) {
    // b = vec(K B) = U_K D_K U_K' B
    CK(L.gemm64(false, nullptr, P->Bm, (double*)P->cpart, nullptr, 0));
    CK(L.combine<double, double>(CM_DK, (double*)P->cpart, nullptr, nullptr, P->tmp64b, P->s2, nullptr));
    CK(L.gemm64(true, nullptr, P->tmp64b, (double*)P->cpart, nullptr, 0));
    CK(L.combine<double, double>(CM_STORE, (double*)P->cpart, nullptr, nullptr, P->tmp64, P->s2, nullptr));
    CK(download(b_out, P->tmp64, nr * sizeof(double), mem, st));
  }
  CK(cudaStreamSynchronize(st));
  return CPHIFI_OK;
}

extern "C" int cphifi_problem_matvec(cphifi_problem* P, int precision, double lambda, double rho,
                                     const double* X, double* Y, int mem) {
  if (!P || !X || !Y) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  const bool gram = (precision & CPHIFI_GRAM_FORM) != 0;
  precision &= ~CPHIFI_GRAM_FORM;
  if (precision < CPHIFI_FP64 || precision > CPHIFI_MIXED_BF16X3)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "unknown precision");
  if (is_tc(precision) && !P->kern->tc)
    return fail(ctx, CPHIFI_E_UNSUPPORTED, "tensor-core products unavailable for this kernel");
  if (precision == CPHIFI_MIXED_BF16X3 && !P->ozb)
    return fail(ctx, CPHIFI_E_UNSUPPORTED, "BF16 slices of U_K unavailable for this kernel");
  Enter guard(ctx);
  int rc;
  if ((rc = precision == CPHIFI_FP64 ? ensure_fp64(P) : ensure_lowp(P)) != CPHIFI_OK) return rc;
  if (gram && (rc = ensure_grams(P, is_lowp(precision), !is_lowp(precision))) != CPHIFI_OK)
    return rc;
  cudaStream_t st = P->st;
  const size_t nr = (size_t)P->n * P->r;
  Launcher L{P, st, nullptr};
  L.gram = gram ? 2 : 0;
  DevScalars h{};
  h.lam = lambda;
  h.rho = rho;
  h.rz = 1.0;
  CK(cudaMemcpyAsync(P->s2, &h, sizeof(DevScalars), cudaMemcpyHostToDevice, st));
  CK(upload(P->tmp64, X, nr * sizeof(double), mem, st));
  // xbar = U_K' X, then the operator in the eigenbasis, then Y = U_K ybar
  CK(L.gemm64(false, nullptr, P->tmp64, (double*)P->cpart, nullptr, 0));
  CK(L.combine<double, double>(CM_STORE, (double*)P->cpart, nullptr, nullptr, P->tmp64b, P->s2, nullptr));
  if (is_lowp(precision)) {
    CK(launch_scale_to<double, float>(P->tmp64b, P->kern->dK, P->n, (int64_t)nr, P->pop32, P->ldt, st));
    if (precision == CPHIFI_MIXED_BF16)
      CK(launch_scale_to<double, __nv_bfloat16>(P->tmp64b, P->kern->dK, P->n, (int64_t)nr, P->pop16,
                                                P->ldt, st));
    CK(L.op_lowp(precision, P->tmp64b, P->y, P->s2, nullptr));
  } else {
    CK(L.opwide(precision == CPHIFI_FP64_EMULATED, CM_APPLY, P->tmp64b, P->y, P->s2, nullptr, 0));
  }
  CK(L.gemm64(true, nullptr, P->y, (double*)P->cpart, nullptr, 0));
  CK(L.combine<double, double>(CM_STORE, (double*)P->cpart, nullptr, nullptr, P->tmp64, P->s2, nullptr));
  CK(download(Y, P->tmp64, nr * sizeof(double), mem, st));
  CK(cudaStreamSynchronize(st));
  return CPHIFI_OK;
}

extern "C" int cphifi_problem_gds(cphifi_problem* P, int precision, const double* Xhat, double* Y1,
                                  int mem) {
  if (!P || !Xhat || !Y1) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  const bool gram = (precision & CPHIFI_GRAM_FORM) != 0;
  precision &= ~CPHIFI_GRAM_FORM;
  if (precision < CPHIFI_FP64 || precision > CPHIFI_MIXED_BF16X3)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "unknown precision");
  Enter guard(ctx);
  int rc;
  if ((rc = precision == CPHIFI_FP64 ? ensure_fp64(P) : ensure_lowp(P)) != CPHIFI_OK) return rc;
  if (gram && (rc = ensure_grams(P, is_lowp(precision), !is_lowp(precision))) != CPHIFI_OK)
    return rc;
  cudaStream_t st = P->st;
  const size_t nr = (size_t)P->n * P->r;
  Launcher L{P, st, nullptr};
  CK(upload(P->xh64, Xhat, nr * sizeof(double), mem, st));
  if (gram && !is_lowp(precision)) {
    CK(L.gram64(P->xh64, P->y164, nullptr, 0));
  } else if (gram) {
    CK(launch_convert<double, float>(P->xh64, P->xh32, (int64_t)nr, st));
    CK(L.gram32(P->xh32, P->y132, nullptr, 0));
    CK(launch_convert<float, double>(P->y132, P->y164, (int64_t)nr, st));
  } else if (precision == CPHIFI_FP64) {
    CK(L.gds64(P->xh64, P->y164, nullptr, 0));
  } else if (precision == CPHIFI_FP64_EMULATED) {
    CK(L.gdsdf(P->xh64, P->y164, nullptr, 0));
  } else {
    CK(launch_convert<double, float>(P->xh64, P->xh32, (int64_t)nr, st));
    CK(L.gds32(P->xh32, P->y132, nullptr, 0));
    CK(launch_convert<float, double>(P->y132, P->y164, (int64_t)nr, st));
  }
  CK(download(Y1, P->y164, nr * sizeof(double), mem, st));
  CK(cudaStreamSynchronize(st));
  return CPHIFI_OK;
}

extern "C" int cphifi_problem_grams(cphifi_problem* P, int precision, double* C, int mem) {
  if (!P || !C) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  if (precision < CPHIFI_FP64 || precision > CPHIFI_MIXED_BF16X3)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "unknown precision");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  Enter guard(ctx);
  const bool lowp = is_lowp(precision);
  int rc;
  if ((rc = precision == CPHIFI_FP64 ? ensure_fp64(P) : ensure_lowp(P)) != CPHIFI_OK) return rc;
  if ((rc = ensure_grams(P, lowp, !lowp)) != CPHIFI_OK) return rc;
  cudaStream_t st = P->st;
  const size_t cnt = (size_t)P->n * P->r * P->r;
  if (!lowp) {
    CK(download(C, P->C64, cnt * sizeof(double), mem, st));
  } else if (mem == CPHIFI_MEM_DEVICE) {
    CK(launch_convert<float, double>(P->C32, C, (int64_t)cnt, st));
  } else {
    std::vector<float> h(cnt);
    CK(cudaMemcpyAsync(h.data(), P->C32, cnt * sizeof(float), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (size_t t = 0; t < cnt; ++t) C[t] = (double)h[t];
  }
  CK(cudaStreamSynchronize(st));
  return CPHIFI_OK;
}

extern "C" int cphifi_problem_precond(cphifi_problem* P, double lambda, double rho, const double* X,
                                      double* Y, int mem) {
  if (!P || !X || !Y) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  if (!(rho > 0.0) || !(lambda >= 0.0)) return fail(ctx, CPHIFI_E_INVALID_ARG, "lambda/rho");
  Enter guard(ctx);
  cudaStream_t st = P->st;
  const size_t nr = (size_t)P->n * P->r;
  Launcher L{P, st, nullptr};
  CK(launch_build_D(P->kern->dK, P->dV, P->n, P->r, P->gamma, lambda, rho, P->D64, P->D32, st));
  CK(upload(P->tmp64, X, nr * sizeof(double), mem, st));
  CK(L.gemm64(false, nullptr, P->tmp64, (double*)P->cpart, nullptr, 0));
  CK(L.combine<double, double>(CM_STORE, (double*)P->cpart, nullptr, nullptr, P->tmp64b, P->s2, nullptr));
  CK(launch_precond_only(P->n, P->r, P->tmp64b, P->tmp64, P->UV, P->D64, st));
  CK(L.gemm64(true, nullptr, P->tmp64, (double*)P->cpart, nullptr, 0));
  CK(L.combine<double, double>(CM_STORE, (double*)P->cpart, nullptr, nullptr, P->tmp64b, P->s2, nullptr));
  CK(download(Y, P->tmp64b, nr * sizeof(double), mem, st));
  CK(cudaStreamSynchronize(st));
  return CPHIFI_OK;
}

extern "C" int cphifi_problem_set_factors(cphifi_problem* P, const double* const* factors,
                                          int mem) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  if (!P->keep_obs) return fail(ctx, CPHIFI_E_INVALID_ARG, "problem created without CPHIFI_KEEP_OBS");
  if (!factors) return fail(ctx, CPHIFI_E_INVALID_ARG, "null factors");
  if (mem != CPHIFI_MEM_HOST && mem != CPHIFI_MEM_DEVICE)
    return fail(ctx, CPHIFI_E_INVALID_ARG, "mem must be HOST or DEVICE");
  for (int m = 0; m < P->d_other; ++m)
    if (!factors[m]) return fail(ctx, CPHIFI_E_INVALID_ARG, "null factor");
  Enter guard(ctx);
  for (int m = 0; m < P->d_other; ++m)
    CK(upload(P->factors[m], factors[m], (size_t)P->sizes[m] * P->r * sizeof(double), mem, P->st));
  return problem_rebuild(P);
}

extern "C" int cphifi_problem_update_factor(cphifi_problem* P, int32_t mode, const double* W,
                                            double* A_out, int mem) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  Enter guard(P->ctx);
  return update_factor(P, mode, W, A_out, mem);
}

extern "C" int cphifi_problem_fit(cphifi_problem* P, const double* W, int mem, double* res2,
                                  double* t2) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  Enter guard(P->ctx);
  return problem_fit(P, W, mem, res2, t2);
}

extern "C" int cphifi_als(cphifi_ctx* ctx, const cphifi_kernel* kern, int32_t d_other,
                          const int64_t* other_sizes, double* const* factors_io, int32_t r,
                          int64_t q, const int32_t* kidx, const int32_t* oidx, const void* vals,
                          uint32_t flags, const cphifi_params* params, int32_t sweeps,
                          double als_tol, int32_t warm, double* W_io, double* err_out,
                          int32_t* sweeps_done, int mem, cphifi_stats* stats) {
  if (!ctx) return CPHIFI_E_INVALID_ARG;
  int rc = check_params(ctx, params);
  if (rc != CPHIFI_OK) return rc;
  if (sweeps < 1 || !W_io || !err_out || !factors_io || !(als_tol >= 0.0))
    return fail(ctx, CPHIFI_E_INVALID_ARG, "bad sweeps, tolerance or output pointers");
  if (sweeps_done) *sweeps_done = 0;
  flags |= CPHIFI_KEEP_OBS |
           (params->precision == CPHIFI_FP64 ? CPHIFI_NEED_FP64 : CPHIFI_NEED_LOWP);
  cphifi_problem* P = nullptr;
  rc = cphifi_problem_create(ctx, kern, d_other, other_sizes, (const double* const*)factors_io, r,
                             q, kidx, oidx, vals, flags, mem, &P);
  if (rc != CPHIFI_OK) return rc;
  Enter guard(ctx);
  const int n = P->n;
  double* Wd = nullptr;   // the current weights on the device
  size_t gw = 0;
  if (pool_alloc(ctx, (size_t)n * r * sizeof(double), (void**)&Wd, &gw) != cudaSuccess) {
    cphifi_problem_destroy(P);
    return fail(ctx, CPHIFI_E_OOM, "weights allocation failed");
  }
  bool have_w = false;
  if (warm) {
    if (upload(Wd, W_io, (size_t)n * r * sizeof(double), mem, P->st) != cudaSuccess) rc = CPHIFI_E_DEVICE;
    have_w = true;
  }
  int s = 0;
  cphifi_stats st_last{};
  for (; rc == CPHIFI_OK && s < sweeps; ++s) {
    // kernel mode (§4): PCG from the previous weights
    rc = solve_prepare(P, params, Wd, CPHIFI_MEM_DEVICE);
    if (rc != CPHIFI_OK) break;
    {
      SolveRun run(P, *params, have_w ? Wd : nullptr, Wd, CPHIFI_MEM_DEVICE, false);
      rc = run.begin();
      while (rc == CPHIFI_OK && run.stage != SolveRun::DONE) {
        if ((rc = run.wait_ready()) != CPHIFI_OK) break;
        rc = run.advance();
      }
      if (rc == CPHIFI_OK) {
        run.fill(&st_last);
        if (run.status != CPHIFI_OK && run.status != CPHIFI_E_NOT_CONVERGED) rc = run.status;
      }
    }
    if (rc != CPHIFI_OK) break;
    have_w = true;
    // finite modes in order (§2)
    for (int m = 0; m < d_other && rc == CPHIFI_OK; ++m)
      rc = update_factor(P, m, Wd, nullptr, CPHIFI_MEM_DEVICE);
    if (rc != CPHIFI_OK) break;
    double r2 = 0.0, t2 = 0.0;
    rc = problem_fit(P, Wd, CPHIFI_MEM_DEVICE, &r2, &t2);
    if (rc != CPHIFI_OK) break;
    err_out[s] = t2 > 0 ? std::sqrt(r2 / t2) : std::sqrt(r2);
    if (sweeps_done) *sweeps_done = s + 1;
    if (als_tol > 0 && s > 0 && std::fabs(err_out[s - 1] - err_out[s]) < als_tol) {
      ++s;
      break;
    }
  }
  if (rc == CPHIFI_OK) {
    if (download(W_io, Wd, (size_t)n * r * sizeof(double), mem, P->st) != cudaSuccess)
      rc = CPHIFI_E_DEVICE;
    for (int m = 0; m < d_other && rc == CPHIFI_OK; ++m)
      if (download(factors_io[m], P->factors[m], (size_t)P->sizes[m] * r * sizeof(double), mem,
                   P->st) != cudaSuccess)
        rc = CPHIFI_E_DEVICE;
    if (cudaStreamSynchronize(P->st) != cudaSuccess) rc = CPHIFI_E_DEVICE;
    if (rc != CPHIFI_OK) fail(ctx, rc, "copying the fitted model out");
  }
  if (stats) *stats = st_last;
  cudaStreamSynchronize(P->st);
  pool_release(ctx, Wd, gw);
  cphifi_problem_destroy(P);
  return rc;
}

extern "C" int cphifi_problem_gram(cphifi_problem* P, double* V, double* DV, double* UV) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  Enter guard(ctx);
  cudaStream_t st = P->st;
  const size_t rr = (size_t)P->r * P->r;
  if (V) CK(cudaMemcpyAsync(V, P->V, rr * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (DV) CK(cudaMemcpyAsync(DV, P->dV, P->r * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (UV) CK(cudaMemcpyAsync(UV, P->UV, rr * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return CPHIFI_OK;
}

extern "C" int cphifi_problem_order(cphifi_problem* P, int32_t* perm, int64_t* row_ptr) {
  if (!P) return CPHIFI_E_INVALID_ARG;
  cphifi_ctx* ctx = P->ctx;
  Enter guard(ctx);
  cudaStream_t st = P->st;
  if (perm) CK(cudaMemcpyAsync(perm, P->perm, P->q * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (row_ptr)
    CK(cudaMemcpyAsync(row_ptr, P->row_ptr, (P->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return CPHIFI_OK;
}
