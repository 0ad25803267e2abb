// cphifi_gds_noalloc: the gather-dot/scatter product (xbar_l = Xhat(i_l,:) .
// Zhat(l,:), Yhat1(i,:) = sum over l with i_l = i of xbar_l Zhat(l,:)), the
// same computation as cphifi_problem_gds in FP64, for callers that must not
// allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not an option, e.g. a
// host thread driving a real-time loop that may not take the allocator's
// locks or wait for its implicit device synchronisation, or an embedding
// runtime that owns all device memory itself and forbids libraries from
// taking more.  Such a caller passes its own inputs and outputs; the working
// memory this computation needs (the piece list, the per-piece partial rows,
// the per-index tickets, an error word) comes from one fixed array compiled
// into this library instead of from the allocator.
//
// The array is `g_noalloc_scratch` below: kNoallocScratchBytes bytes of
// device memory in every GPU that loads the library, held until the process
// exits.  It is shared by every call on a device, so two calls whose work
// overlaps on the GPU (different streams, or different host threads) race
// and both results are undefined; serialise them on one stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "cphifi.h"
#include "launch.h"

namespace cphifi {
namespace {

constexpr int kNoallocMaxN = 16384;       // kernel-mode size limit
constexpr int kNoallocMaxRank = 64;       // rank limit
constexpr int kNoallocMaxWarps = 4096;    // warps of the product (<= 16 per SM)
constexpr int64_t kNoallocMaxPieces = (int64_t)kNoallocMaxN + kNoallocMaxWarps + 1;

// Byte offsets of the pieces of the scratch array (each 256-byte aligned).
constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffErr = 0;  // error word: nonzero = row_ptr is not a CSR of q
constexpr size_t kOffCount = kOffErr + 256;
constexpr size_t kOffFirst = kOffCount + al(sizeof(int32_t) * kNoallocMaxN);
constexpr size_t kOffTicket = kOffFirst + al(sizeof(int32_t) * (kNoallocMaxN + 1));
constexpr size_t kOffSeg = kOffTicket + al(sizeof(unsigned) * kNoallocMaxN);
constexpr size_t kOffBeg = kOffSeg + al(sizeof(int32_t) * kNoallocMaxPieces);
constexpr size_t kOffEnd = kOffBeg + al(sizeof(int32_t) * kNoallocMaxPieces);
constexpr size_t kOffWarp = kOffEnd + al(sizeof(int32_t) * kNoallocMaxPieces);
constexpr size_t kOffScan = kOffWarp + al(sizeof(int32_t) * (kNoallocMaxWarps + 1));
constexpr size_t kScanBytes = al(sizeof(int64_t) * (kNoallocMaxN / 2048 + 2));
constexpr size_t kOffPartial = kOffScan + kScanBytes;
constexpr size_t kNoallocScratchBytes =
    kOffPartial + al(sizeof(double) * kNoallocMaxPieces * kNoallocMaxRank);

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// The caller's row_ptr must be a CSR of q observations: row_ptr[0] = 0,
// non-decreasing, row_ptr[n] = q.  Anything else sets *err, and every later
// kernel of the call then returns without touching memory (a bad row_ptr
// would otherwise index past the piece arrays and past Zhat); the last kernel
// fills Y1 with NaN so that the caller sees the failure.
__global__ void noalloc_check_csr_kernel(const int64_t* __restrict__ row_ptr, int n, int64_t q,
                                         int* err) {
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
    const int64_t v = row_ptr[i];
    if (i == 0 && v != 0) bad = 1;
    if (i == n && v != q) bad = 1;
    if (i < n && row_ptr[i + 1] < v) bad = 1;
  }
  if (bad) atomicOr(err, 1);
}

// warp_first for the no-allocation path: like launch_warp_first, but the
// number of pieces is read on the device (seg_first[n], clamped to the
// scratch array's piece capacity) so the host never waits for it.
__global__ void noalloc_warp_first_kernel(const int32_t* __restrict__ pbeg,
                                          const int32_t* __restrict__ seg_first, int n,
                                          int64_t L, int W, int32_t* warp_first,
                                          const int* gate) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > W || *gate) return;
  const int npieces = (int)min((int64_t)seg_first[n], kNoallocMaxPieces);
  if (w == W) { warp_first[W] = npieces; return; }
  const int64_t v = (int64_t)w * L;
  int lo = 0, hi = npieces;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)pbeg[mid] < v) lo = mid + 1; else hi = mid;
  }
  warp_first[w] = lo;
}

// Y1 = NaN when the CSR check failed.
__global__ void noalloc_flag_output_kernel(const int* gate, int64_t count, double* Y) {
  if (!*gate) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    Y[t] = __longlong_as_double(0x7ff8000000000000LL);
}

// The gather-dot/scatter of gds_kernel (Eqs. vl and yhat1), FP64, reading Zhat
// in the caller's plain column-major layout (Zhat(l, j) at j*ldz + l).
template <int RP>
__global__ void __launch_bounds__(256)
noalloc_gds_kernel(PieceList pl, const double* __restrict__ Z, int64_t ldz, int r,
                   const double* __restrict__ Xh, int64_t ldx, double* __restrict__ partial,
                   double* __restrict__ Y, int64_t ldy, const int* gate) {
  __shared__ double xs[8][RP];
  if (*gate) return;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int w = gw; w < pl.nwarps; w += nwarps) {
    const int p_end = pl.warp_first[w + 1];
    for (int p = pl.warp_first[w]; p < p_end; ++p) {
      const int seg = pl.seg[p];
      const int b = pl.beg[p], e = pl.end[p];
      __syncwarp();
      for (int j = lane; j < RP; j += 32) xs[wib][j] = j < r ? Xh[(int64_t)j * ldx + seg] : 0.0;
      __syncwarp();
      double acc[RP];
#pragma unroll
      for (int j = 0; j < RP; ++j) acc[j] = 0.0;
      for (int l = b + lane; l < e; l += 32) {
        double xb = 0.0;
#pragma unroll
        for (int j = 0; j < RP; ++j)
          if (j < r) xb = fma(xs[wib][j], Z[(int64_t)j * ldz + l], xb);
#pragma unroll
        for (int j = 0; j < RP; ++j)
          if (j < r) acc[j] = fma(xb, Z[(int64_t)j * ldz + l], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < RP; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
      const int np = pl.seg_count[seg];
      if (np == 1) {
#pragma unroll
        for (int j = 0; j < RP; ++j)
          if ((j & 31) == lane && j < r) Y[(int64_t)j * ldy + seg] = acc[j];
      } else {
#pragma unroll
        for (int j = 0; j < RP; ++j)
          if ((j & 31) == lane && j < r) partial[(int64_t)p * RP + j] = acc[j];
        __threadfence();
        __syncwarp();
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(&pl.seg_ticket[seg], 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t == (unsigned)(np - 1)) {
          __threadfence();
          const int f = pl.seg_first[seg];
          for (int j = lane; j < r; j += 32) {
            double s = 0.0;
            for (int k = 0; k < np; ++k) s += __ldcg(&partial[(int64_t)(f + k) * RP + j]);
            Y[(int64_t)j * ldy + seg] = s;
          }
          if (lane == 0) pl.seg_ticket[seg] = 0u;
        }
      }
    }
  }
}

namespace {

struct DeviceSlot {
  bool ready = false;
  unsigned char* base = nullptr;
  int num_sms = 0;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;

// The device address of the scratch array (the host-side name
// g_noalloc_scratch is only a stand-in for it) and the SM count, looked up
// with the device current on its first successful call and kept from then
// on.  A failed lookup is not cached: the next call tries again.
cudaError_t device_slot(int dev, DeviceSlot* out) {
  std::lock_guard<std::mutex> lock(g_slots_mu);
  DeviceSlot* s = &g_slots[dev];
  if (!s->ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    s->base = (unsigned char*)ptr;
    s->num_sms = sms;
    s->ready = true;
  }
  *out = *s;
  return cudaSuccess;
}

int reject(const char** msg, const char* text) {
  if (msg) *msg = text;
  return CPHIFI_E_INVALID_ARG;
}

}  // namespace
}  // namespace cphifi

using namespace cphifi;

extern "C" int cphifi_gds_noalloc(int32_t n, int32_t r, int64_t q, const int64_t* row_ptr,
                                  const double* zhat, int64_t ldz, const double* Xhat,
                                  double* Y1, void* stream, const char** err_msg) {
  if (err_msg) *err_msg = "ok";
  if (n < 1 || n > kNoallocMaxN)
    return reject(err_msg, "cphifi_gds_noalloc: n must be in [1, 16384]");
  if (r < 1 || r > kNoallocMaxRank)
    return reject(err_msg, "cphifi_gds_noalloc: r must be in [1, 64]");
  if (q < 0 || q >= (int64_t(1) << 31))
    return reject(err_msg, "cphifi_gds_noalloc: q must be in [0, 2^31)");
  if (ldz < q) return reject(err_msg, "cphifi_gds_noalloc: ldz must be >= q");
  if (!row_ptr || !Xhat || !Y1 || (q > 0 && !zhat))
    return reject(err_msg, "cphifi_gds_noalloc: null device pointer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    if (err_msg) *err_msg = "cphifi_gds_noalloc: no usable current CUDA device";
    return CPHIFI_E_DEVICE;
  }
  DeviceSlot slot;
  if (device_slot(dev, &slot) != cudaSuccess) {
    if (err_msg) *err_msg = "cphifi_gds_noalloc: cudaGetSymbolAddress of the scratch array failed";
    return CPHIFI_E_DEVICE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = slot.base;
  int* gate = (int*)(base + kOffErr);
  int32_t* seg_count = (int32_t*)(base + kOffCount);
  int32_t* seg_first = (int32_t*)(base + kOffFirst);
  unsigned* seg_ticket = (unsigned*)(base + kOffTicket);
  int32_t* pseg = (int32_t*)(base + kOffSeg);
  int32_t* pbeg = (int32_t*)(base + kOffBeg);
  int32_t* pend = (int32_t*)(base + kOffEnd);
  int32_t* warp_first = (int32_t*)(base + kOffWarp);
  void* scan_tmp = base + kOffScan;
  double* partial = (double*)(base + kOffPartial);

  int64_t W64 = (q + 63) / 64;
  const int64_t wcap = std::min<int64_t>((int64_t)slot.num_sms * 16, kNoallocMaxWarps);
  if (W64 > wcap) W64 = wcap;
  if (W64 < 1) W64 = 1;
  const int W = (int)W64;
  const int64_t L = std::max<int64_t>(1, (q + W - 1) / W);

  cudaError_t e = cudaSuccess;
  // The error word and the tickets must start at zero: the array keeps what
  // the last call left (the last piece of an index resets its own ticket, but
  // a call cut short by a failed check leaves stale counts behind).
  e = cudaMemsetAsync(base, 0, kOffCount, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(seg_ticket, 0, sizeof(unsigned) * n, st);
  if (e == cudaSuccess) {
    noalloc_check_csr_kernel<<<(n + 1 + 255) / 256, 256, 0, st>>>(row_ptr, n, q, gate);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_piece_counts(row_ptr, n, L, seg_count, gate, st);
  if (e == cudaSuccess) e = exclusive_scan_i32(seg_count, seg_first, n, scan_tmp, kScanBytes, st);
  if (e == cudaSuccess)
    e = launch_piece_fill(row_ptr, n, L, seg_first, seg_count, pseg, pbeg, pend, gate, st);
  if (e == cudaSuccess) {
    noalloc_warp_first_kernel<<<(W + 1 + 255) / 256, 256, 0, st>>>(pbeg, seg_first, n, L, W,
                                                                  warp_first, gate);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    PieceList pl{pseg, pbeg, pend, seg_first, seg_count, seg_ticket, warp_first,
                 (int)kNoallocMaxPieces, W};
    const int blocks = (W + 7) / 8;
    if (r <= 8)
      noalloc_gds_kernel<8><<<blocks, 256, 0, st>>>(pl, zhat, ldz, r, Xhat, n, partial, Y1, n,
                                                    gate);
    else if (r <= 16)
      noalloc_gds_kernel<16><<<blocks, 256, 0, st>>>(pl, zhat, ldz, r, Xhat, n, partial, Y1, n,
                                                     gate);
    else if (r <= 32)
      noalloc_gds_kernel<32><<<blocks, 256, 0, st>>>(pl, zhat, ldz, r, Xhat, n, partial, Y1, n,
                                                     gate);
    else
      noalloc_gds_kernel<64><<<blocks, 256, 0, st>>>(pl, zhat, ldz, r, Xhat, n, partial, Y1, n,
                                                     gate);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int64_t count = (int64_t)n * r;
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, 1024);
    noalloc_flag_output_kernel<<<blocks, 256, 0, st>>>(gate, count, Y1);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    if (err_msg) *err_msg = "cphifi_gds_noalloc: a CUDA launch failed";
    return CPHIFI_E_DEVICE;
  }
  return CPHIFI_OK;
}
