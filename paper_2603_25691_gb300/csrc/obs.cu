// Observation-side kernels: validation, the stable sort by kernel index, the
// CSR row pointer, the piece list, Zhat (Eq. zhat, §4.2) and the fused
// gather-dot/scatter of the matrix-free product (Eqs. vl and yhat1, §4.4.1).
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "gds.cuh"
#include "launch.h"

namespace cphifi {

// ----------------------------------------------------------- validation ---
// Kernel indices in [0, n) (bit 1 of *err), and non-decreasing when the
// caller declared them sorted (bit 4).  The other modes' indices and the
// values are checked by the Zhat build, which reads them anyway.
__global__ void validate_kidx_kernel(const int32_t* __restrict__ kidx, int64_t q, int n,
                                     bool sorted, int* err) {
  int bad = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < q;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = kidx[l];
    if (k < 0 || k >= n) bad |= 1;
    if (sorted && l + 1 < q && kidx[l + 1] < k) bad |= 4;
  }
  if (bad) atomicOr(err, bad);
}

cudaError_t launch_validate_kidx(const int32_t* kidx, int64_t q, int n, bool sorted, int* err,
                                 cudaStream_t st) {
  if (q == 0) return cudaSuccess;
  const int blocks = (int)((q + 255) / 256 < 4096 ? (q + 255) / 256 : 4096);
  validate_kidx_kernel<<<blocks, 256, 0, st>>>(kidx, q, n, sorted, err);
  return cudaGetLastError();
}

__global__ void validate_dense_kernel(const double* __restrict__ a, int64_t count, int* err) {
  int bad = 0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < count;
       l += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[l])) bad = 2;
  if (bad) atomicOr(err, bad);
}

cudaError_t launch_validate_dense(const double* a, int64_t count, int* err, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int blocks = (int)((count + 255) / 256 < 2048 ? (count + 255) / 256 : 2048);
  validate_dense_kernel<<<blocks, 256, 0, st>>>(a, count, err);
  return cudaGetLastError();
}

__global__ void iota_kernel(int32_t* v, int64_t q) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < q;
       l += (int64_t)gridDim.x * blockDim.x)
    v[l] = (int32_t)l;
}

cudaError_t launch_iota(int32_t* v, int64_t q, cudaStream_t st) {
  if (q == 0) return cudaSuccess;
  const int blocks = (int)((q + 255) / 256 < 4096 ? (q + 255) / 256 : 4096);
  iota_kernel<<<blocks, 256, 0, st>>>(v, q);
  return cudaGetLastError();
}

// ------------------------------------------------------ exclusive scan ----
// Three-phase scan of int32 counts: per-chunk sums, a scan of the chunk sums
// by one block, then per-chunk scans with the chunk offset.  out[n] = total.
constexpr int kScanChunk = 2048;  // 256 threads x 8 items

__global__ void scan_chunk_sums(const int32_t* __restrict__ in, int64_t n, int64_t* sums) {
  __shared__ double sm[32];
  const int64_t base = blockIdx.x * (int64_t)kScanChunk;
  double v[1] = {0.0};
  for (int k = threadIdx.x; k < kScanChunk; k += blockDim.x) {
    const int64_t i = base + k;
    if (i < n) v[0] += (double)in[i];
  }
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) sums[blockIdx.x] = (int64_t)v[0];
}

__global__ void scan_sums_serial(int64_t* sums, int64_t nchunks) {
  // One block: exclusive scan of the chunk sums in place, tile by tile.
  __shared__ int64_t tile[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t t0 = 0; t0 < nchunks; t0 += 1024) {
    const int64_t i = t0 + threadIdx.x;
    const int64_t v = i < nchunks ? sums[i] : 0;
    tile[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int64_t add = threadIdx.x >= o ? tile[threadIdx.x - o] : 0;
      __syncthreads();
      tile[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nchunks) sums[i] = carry + tile[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += tile[1023];
    __syncthreads();
  }
}

__global__ void scan_chunks_final(const int32_t* __restrict__ in, int64_t n,
                                  const int64_t* __restrict__ sums, int32_t* out) {
  __shared__ int64_t ts[256];
  const int64_t base = blockIdx.x * (int64_t)kScanChunk + threadIdx.x * 8;
  int64_t loc[8];
  int64_t run = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t i = base + k;
    loc[k] = run;
    run += i < n ? in[i] : 0;
  }
  ts[threadIdx.x] = run;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int64_t add = threadIdx.x >= o ? ts[threadIdx.x - o] : 0;
    __syncthreads();
    ts[threadIdx.x] += add;
    __syncthreads();
  }
  const int64_t off = sums[blockIdx.x] + ts[threadIdx.x] - run;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t i = base + k;
    if (i < n) out[i] = (int32_t)(off + loc[k]);
    if (i == n - 1) out[n] = (int32_t)(off + loc[k] + in[i]);
  }
}

size_t exclusive_scan_tmp_bytes(int64_t n) {
  return (size_t)((n + kScanChunk - 1) / kScanChunk + 1) * sizeof(int64_t);
}

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp,
                               size_t tmp_bytes, cudaStream_t st) {
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), st);
  const int64_t nchunks = (n + kScanChunk - 1) / kScanChunk;
  if (tmp_bytes < exclusive_scan_tmp_bytes(n)) return cudaErrorInvalidValue;
  int64_t* sums = (int64_t*)tmp;
  scan_chunk_sums<<<(unsigned)nchunks, 256, 0, st>>>(in, n, sums);
  scan_sums_serial<<<1, 1024, 0, st>>>(sums, nchunks);
  scan_chunks_final<<<(unsigned)nchunks, 256, 0, st>>>(in, n, sums, out);
  return cudaGetLastError();
}

// ------------------------------------------------------- LSD radix sort ---
// 8-bit digits; a tile of 4096 keys per block (8 warps x 16 rounds x 32).
// The scatter ranks each key among equal digits of its tile in input order
// (warp match + per-warp counters + a scan over warps), so every pass is
// stable and so is the whole sort.
constexpr int kRsTile = 4096;

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t q, int shift,
                                  uint32_t* hist, int ntiles) {
  __shared__ uint32_t h[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kRsTile;
  for (int k = threadIdx.x; k < kRsTile; k += blockDim.x) {
    const int64_t l = base + k;
    if (l < q) atomicAdd(&h[(keys[l] >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                     uint32_t* __restrict__ kout, int32_t* __restrict__ vout,
                                     int64_t q, int shift, const int32_t* __restrict__ offs,
                                     int ntiles) {
  __shared__ uint32_t wcount[8][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < 8 * 256; t += blockDim.x) (&wcount[0][0])[t] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)kRsTile + w * 512;
  uint32_t key[16], rank[16];
  int32_t val[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t l = base + k * 32 + lane;
    const bool valid = l < q;
    key[k] = valid ? kin[l] : 0u;
    val[k] = valid ? vin[l] : 0;
    const uint32_t d = valid ? ((key[k] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned lower = peers & ((1u << lane) - 1u);
    const uint32_t before = valid ? wcount[w][d] : 0u;
    __syncwarp();
    if (valid && lower == 0u) wcount[w][d] = before + __popc(peers);
    __syncwarp();
    rank[k] = before + __popc(lower);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    uint32_t run = 0;
    for (int ww = 0; ww < 8; ++ww) {
      const uint32_t c = wcount[ww][d];
      wcount[ww][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t l = base + k * 32 + lane;
    if (l < q) {
      const uint32_t d = (key[k] >> shift) & 255u;
      const int64_t pos = (int64_t)offs[(int64_t)d * ntiles + blockIdx.x] + wcount[w][d] + rank[k];
      kout[pos] = key[k];
      vout[pos] = val[k];
    }
  }
}

size_t radix_sort_tmp_bytes(int64_t q) {
  const int64_t ntiles = (q + kRsTile - 1) / kRsTile;
  const int64_t nh = 256 * ntiles;
  size_t b = 0;
  b += (size_t)q * sizeof(uint32_t) + 256;        // alternate keys
  b += (size_t)q * sizeof(int32_t) + 256;         // alternate values
  b += (size_t)nh * sizeof(int32_t) + 256;        // histogram
  b += (size_t)(nh + 1) * sizeof(int32_t) + 256;  // offsets
  b += exclusive_scan_tmp_bytes(nh) + 256;
  return b;
}

static inline char* align256(char* p) {
  return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
}

cudaError_t radix_sort_pairs(uint32_t* keys, int32_t* vals, int64_t q, int key_bits,
                             void* tmp, cudaStream_t st) {
  if (q <= 1) return cudaSuccess;
  const int64_t ntiles = (q + kRsTile - 1) / kRsTile;
  const int64_t nh = 256 * ntiles;
  char* p = align256((char*)tmp);
  uint32_t* k2 = (uint32_t*)p; p = align256(p + q * sizeof(uint32_t));
  int32_t* v2 = (int32_t*)p; p = align256(p + q * sizeof(int32_t));
  uint32_t* hist = (uint32_t*)p; p = align256(p + nh * sizeof(int32_t));
  int32_t* offs = (int32_t*)p; p = align256(p + (nh + 1) * sizeof(int32_t));
  void* scan_tmp = p;
  const int passes = (key_bits + 7) / 8;
  uint32_t *ka = keys, *kb = k2;
  int32_t *va = vals, *vb = v2;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 8 * ps;
    radix_hist_kernel<<<(unsigned)ntiles, 256, 0, st>>>(ka, q, shift, hist, (int)ntiles);
    cudaError_t e = exclusive_scan_i32((const int32_t*)hist, offs, nh, scan_tmp,
                                       exclusive_scan_tmp_bytes(nh), st);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<(unsigned)ntiles, 256, 0, st>>>(ka, va, kb, vb, q, shift, offs, (int)ntiles);
    uint32_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, q * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, va, q * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  }
  return cudaGetLastError();
}

// ------------------------------------------------- CSR and piece lists ----
__global__ void row_ptr_kernel(const uint32_t* __restrict__ keys, int64_t q, int n,
                               int64_t* row_ptr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  int64_t lo = 0, hi = q;  // first position with key >= i
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < (uint32_t)i) lo = mid + 1; else hi = mid;
  }
  row_ptr[i] = lo;
}

cudaError_t launch_row_ptr(const uint32_t* sorted_keys, int64_t q, int n, int64_t* row_ptr,
                           cudaStream_t st) {
  row_ptr_kernel<<<(n + 1 + 255) / 256, 256, 0, st>>>(sorted_keys, q, n, row_ptr);
  return cudaGetLastError();
}

// Pieces are the pieces of kernel-index segments cut at multiples of L, the
// observation range of one warp: every warp then owns exactly L sorted
// observations (the last one fewer) whatever the segment lengths are.
__global__ void piece_counts_kernel(const int64_t* __restrict__ row_ptr, int n, int64_t L,
                                    int32_t* seg_count, const int* gate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (gate && *gate)) return;
  const int64_t b = row_ptr[i], e = row_ptr[i + 1];
  seg_count[i] = e > b ? (int32_t)((e - 1) / L - b / L + 1) : 1;
}

cudaError_t launch_piece_counts(const int64_t* row_ptr, int n, int64_t L, int32_t* seg_count,
                                const int* gate, cudaStream_t st) {
  piece_counts_kernel<<<(n + 255) / 256, 256, 0, st>>>(row_ptr, n, L, seg_count, gate);
  return cudaGetLastError();
}

__global__ void piece_fill_kernel(const int64_t* __restrict__ row_ptr, int n, int64_t L,
                                  const int32_t* __restrict__ seg_first,
                                  const int32_t* __restrict__ seg_count, int32_t* pseg,
                                  int32_t* pbeg, int32_t* pend, const int* gate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (gate && *gate)) return;
  const int64_t b = row_ptr[i], e = row_ptr[i + 1];
  const int c = seg_count[i];
  const int64_t k0 = b / L;
  for (int k = 0; k < c; ++k) {
    const int p = seg_first[i] + k;
    int64_t pb = (k0 + k) * L, pe = pb + L;
    if (pb < b) pb = b;
    if (pe > e) pe = e;
    if (e == b) pb = pe = b;
    pseg[p] = i;
    pbeg[p] = (int32_t)pb;
    pend[p] = (int32_t)pe;
  }
}

cudaError_t launch_piece_fill(const int64_t* row_ptr, int n, int64_t L, const int32_t* seg_first,
                              const int32_t* seg_count, int32_t* pseg, int32_t* pbeg,
                              int32_t* pend, const int* gate, cudaStream_t st) {
  piece_fill_kernel<<<(n + 255) / 256, 256, 0, st>>>(row_ptr, n, L, seg_first, seg_count, pseg,
                                                     pbeg, pend, gate);
  return cudaGetLastError();
}

// warp_first[w] = first piece starting at or after w*L (w < W); warp_first[W]
// = npieces, so warp w owns pieces [warp_first[w], warp_first[w+1]).  With
// np_dev set, npieces is read from the device (the piece-count scan's total,
// clamped to the allocated npieces) instead.
__global__ void warp_first_kernel(const int32_t* __restrict__ pbeg, int npieces,
                                  const int32_t* np_dev, int64_t L, int W, int32_t* warp_first,
                                  const int* gate) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > W || (gate && *gate)) return;
  if (np_dev) npieces = min(npieces, *np_dev);
  if (w == W) { warp_first[W] = npieces; return; }
  const int64_t v = (int64_t)w * L;
  int lo = 0, hi = npieces;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)pbeg[mid] < v) lo = mid + 1; else hi = mid;
  }
  warp_first[w] = lo;
}

cudaError_t launch_warp_first(const int32_t* pbeg, int npieces, const int32_t* np_dev, int64_t L,
                              int W, int32_t* warp_first, const int* gate, cudaStream_t st) {
  warp_first_kernel<<<(W + 1 + 255) / 256, 256, 0, st>>>(pbeg, npieces, np_dev, L, W,
                                                         warp_first, gate);
  return cudaGetLastError();
}

// -------------------------------------------------------------- Zhat ------
// Zhat(s, j) = prod_m A_m(oidx[perm[s], m], j) for the s-th observation in the
// sorted order (Eq. zhat), computed in double-float arithmetic and stored as an
// unevaluated sum of two FP32 numbers hi + lo (|z - hi - lo| <= 2^-48 |z|):
// hi alone is the FP32 operator's Zhat, hi + lo the FP64 one (and/or the FP64
// value itself).  Storage is in tiles of 32 observations (zidx in launch.h),
// so the 32 x r values a warp round reads form one contiguous block.
//
// The pass that builds Zhat also forms the sparse MTTKRP B(i,:) =
// sum_{i_l = i} t_l Zhat(l,:) (§4, the right-hand side), FP64-accurate, with
// the piece decomposition and deterministic combine of the gather-dot/scatter
// below (zhat_mttkrp_kernel).

// Eight consecutive floats from read-only global memory in one 256-bit load
// (sm_100 and later); p must be 32-byte aligned.  A lane's 32-byte sector
// then takes one load instead of two: the factor-row gathers of the Zhat
// build are bound by the L1 data stage.
__device__ __forceinline__ void ldg_v8(const float* p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7])
      : "l"(p));
}

// ------------------------------------------------ gather-dot / scatter ----
// One launch over the virtual warps of the piece decomposition; the per-warp
// work is gds_warp_range (gds.cuh).  Warps draw their ranges from pl.wctr
// when it is set (dynamic assignment), else take w = gw + k nwarps.
template <int MODE, int RP, int LPO, bool WTS>
__global__ void __launch_bounds__(256, 2) gds_kernel(PieceList pl, const float* __restrict__ zhi,
                                                  const float* __restrict__ zlo,
                                                  const double* __restrict__ z64, int r,
                                                  const typename GdsTypes<MODE>::IO* __restrict__ Xh,
                                                  int64_t xld,
                                                  typename GdsTypes<MODE>::IO* __restrict__ partial,
                                                  typename GdsTypes<MODE>::IO* __restrict__ Y,
                                                  int64_t yld, const DevScalars* skip,
                                                  const double* __restrict__ wts,
                                                  const int32_t* __restrict__ wperm,
                                                  const float2* __restrict__ wdf,
                                                  const int* gate) {
  using Acc = typename GdsTypes<MODE>::Acc;
  (void)zlo;  // the lo block sits inside zhi's tiles (+32 r)
  if (dev_skip(skip) || (gate && *gate)) return;
  __shared__ Acc xs[8][RP];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  auto draw = [&]() -> int {
    unsigned v = 0;
    if (lane == 0) v = atomicAdd(&pl.wctr[0], 1u);
    return (int)__shfl_sync(0xffffffffu, v, 0);
  };
  for (int w = pl.wctr ? draw() : gw; w < pl.nwarps; w = pl.wctr ? draw() : w + nwarps)
    gds_warp_range<MODE, RP, LPO, WTS>(pl, w, zhi, z64, r, Xh, xld, GdsXsrc(), partial, Y, yld,
                                       wts, wperm, wdf, xs[wib]);
  if (pl.wctr && lane == 0) {  // the last warp out resets the counters
    __threadfence();
    if (atomicAdd(&pl.wctr[1], 1u) == (unsigned)nwarps - 1) {
      pl.wctr[0] = 0u;
      pl.wctr[1] = 0u;
      __threadfence();
    }
  }
}

struct GdsWeights {
  const double* wts = nullptr;    // non-null: weights mode (FP64 weights, wperm order)
  const int32_t* wperm = nullptr;
  const float2* wdf = nullptr;    // double-float weights in the sorted order (GDS_DF)
  const int* gate = nullptr;
};

template <int MODE, int RP, int LPO>
static cudaError_t gds_dispatch(const PieceList& pl, const float* zhi, const float* zlo,
                                const double* z64, int r, const typename GdsTypes<MODE>::IO* Xh,
                                int64_t xld, typename GdsTypes<MODE>::IO* partial,
                                typename GdsTypes<MODE>::IO* Y, int64_t yld,
                                const DevScalars* skip, cudaStream_t st,
                                const GdsWeights& wt = GdsWeights()) {
  const int blocks = (pl.nwarps + 7) / 8;
  if (wt.wts || wt.wdf)
    gds_kernel<MODE, RP, LPO, true><<<blocks, 256, 0, st>>>(pl, zhi, zlo, z64, r, Xh, xld, partial,
                                                            Y, yld, skip, wt.wts, wt.wperm,
                                                            wt.wdf, wt.gate);
  else
    gds_kernel<MODE, RP, LPO, false><<<blocks, 256, 0, st>>>(pl, zhi, zlo, z64, r, Xh, xld,
                                                             partial, Y, yld, skip, nullptr,
                                                             nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

// Lanes per observation keep the per-lane registers (RP/LPO values of the
// row and of the accumulator) within budget.  At n = 8000, q = 5e7, r = 40:
// the FP32 pass takes 1.37 ms with its 40-column instance against 1.48 ms
// with 48 columns; the FP64 pass also has one (the FP64 solve 8.4 -> 8.8
// solves/s).  The double-float pass keeps 48 columns: with 40 (4 lanes per
// observation) it ran 2.96 against 3.32 ms alone but 4.6 against 3.9 ms as
// the true residual inside a solve, and 8 lanes per observation took 4.1 ms
// alone.
template <int MODE>
static cudaError_t gds_by_rank(const PieceList& pl, const float* zhi, const float* zlo,
                               const double* z64, int r, const typename GdsTypes<MODE>::IO* Xh,
                               int64_t xld, typename GdsTypes<MODE>::IO* partial,
                               typename GdsTypes<MODE>::IO* Y, int64_t yld,
                               const DevScalars* skip, cudaStream_t st,
                               const GdsWeights& wt = GdsWeights()) {
  if (pl.npieces == 0 || pl.nwarps == 0) return cudaSuccess;
  constexpr bool wide = MODE != GDS_F32;
  if (r <= 8) return gds_dispatch<MODE, 8, 1>(pl, zhi, zlo, z64, r, Xh, xld, partial, Y, yld, skip, st, wt);
  if (r <= 16) return gds_dispatch<MODE, 16, 1>(pl, zhi, zlo, z64, r, Xh, xld, partial, Y, yld, skip, st, wt);
  if (r <= 32) return gds_dispatch<MODE, 32, wide ? 2 : 1>(pl, zhi, zlo, z64, r, Xh, xld, partial, Y, yld, skip, st, wt);
  if constexpr (MODE != GDS_DF) {
    if (r <= 40) return gds_dispatch<MODE, 40, wide ? 4 : 1>(pl, zhi, zlo, z64, r, Xh, xld, partial, Y, yld, skip, st, wt);
  }
  if (r <= 48) return gds_dispatch<MODE, 48, wide ? 4 : 1>(pl, zhi, zlo, z64, r, Xh, xld, partial, Y, yld, skip, st, wt);
  if (r <= 64) return gds_dispatch<MODE, 64, wide ? 4 : 2>(pl, zhi, zlo, z64, r, Xh, xld, partial, Y, yld, skip, st, wt);
  return cudaErrorInvalidValue;
}

// ------------------------------------------ fused Zhat build + MTTKRP ----
// Zhat and B(i,:) = sum_{i_l = i} t_l Zhat(l,:) (§4, the right-hand side) in
// one pass: warp w takes the pieces of its range of sorted observations
// (the gather-dot/scatter decomposition, here with more and shorter ranges),
// builds each 32-observation tile of a piece column group by column group as
// the build kernel does (one lane per observation, double-float products of
// the factor rows, the FP32 pair and/or FP64 stored), and folds t_l Zhat(l,:)
// into the piece's row sum: the 4 columns of a group are summed over the 32
// lanes by a reduce-scatter (lanes exchange halves of the group, then
// butterfly: 12 shuffles, 6 double-float additions per lane), and 4 lanes add
// the tile's 4 column sums into the warp's row in shared memory.  The rows
// are written as the gather-dot/scatter writes them (a kernel index split
// over pieces: partial rows, the last piece adds them in piece order), so B is
// deterministic, and Zhat is never read back.
__device__ __forceinline__ df shfl_xor_df(df v, int m) {
  return df{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

template <bool WHI, bool W64>
__global__ void __launch_bounds__(256, 3)
zhat_mttkrp_kernel(PieceList pl, int64_t q, const int32_t* __restrict__ perm,
                   const int32_t* __restrict__ oidx, int d_other,
                   const float* const* __restrict__ fhl, const int64_t* __restrict__ sizes, int r,
                   float* __restrict__ zhi, double* __restrict__ z64,
                   const double* __restrict__ vals, double* __restrict__ partial,
                   double* __restrict__ B, int64_t ldb, int* err, const int* gate, int w_begin,
                   int w_end) {
  if (gate && *gate) return;  // invalid input found earlier: touch nothing
  __shared__ df bacc[8][64];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  bool vec = (r % 4 == 0);
  for (int m = 0; m < d_other; ++m)
    vec = vec && ((reinterpret_cast<uintptr_t>(fhl[m]) & 31) == 0);
  // reduce-scatter roles: after it, lanes 8c..8c+7 hold column c of a group
  const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
  const int col = (up16 ? 2 : 0) + (up8 ? 1 : 0);
  int bad = 0;
  auto draw = [&]() -> int {
    unsigned v = 0;
    if (lane == 0) v = atomicAdd(&pl.wctr[0], 1u);
    return (int)__shfl_sync(0xffffffffu, v, 0);
  };
  // this launch's virtual warps: [w_begin, w_end) of the decomposition
  for (int w = w_begin + draw(); w < w_end; w = w_begin + draw()) {
    const int p_end = pl.warp_first[w + 1];
    for (int p = pl.warp_first[w]; p < p_end; ++p) {
      const int seg = pl.seg[p];
      const int64_t b = pl.beg[p], e = pl.end[p];
      __syncwarp();
      for (int j = lane; j < 64; j += 32) bacc[wib][j] = df{0.f, 0.f};
      __syncwarp();
      for (int64_t tile = b >> 5; e > b && tile <= (e - 1) >> 5; ++tile) {
        const int64_t l = tile * 32 + lane;
        const bool act = l >= b && l < e;
        const int64_t src = act ? (perm ? (int64_t)perm[l] : l) : 0;
        const double tv = act ? vals[src] : 0.0;
        bad |= isfinite(tv) ? 0 : 2;
        const df t = df_from_double(tv);
        const int32_t* im = oidx + src * d_other;
        bool ok = act;
        for (int m = 0; act && m < d_other; ++m) {
          const int32_t v = __ldg(im + m);
          ok = ok && v >= 0 && v < sizes[m];
        }
        bad |= (act && !ok) ? 1 : 0;
        const int64_t base = tile * 64 * (int64_t)r + (l & 31);    // hi tile; lo = +32 r
        const int64_t base64 = tile * 32 * (int64_t)r + (l & 31);  // FP64 copy
        // the 4 columns j0..j0+3 of Zhat(l, :): stored, then t_l Zhat(l, j0..j0+3)
        // summed over the tile's lanes into the piece's row
        auto emit = [&](int j0, df (&z)[4]) {
          if (ok) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = j0 + u;
              if (j < r) {
                if constexpr (WHI) {
                  __stcs(zhi + base + 32 * (int64_t)j, z[u].hi);
                  __stcs(zhi + base + 32 * (int64_t)j + 32 * r, z[u].lo);
                }
                if constexpr (W64) __stcs(z64 + base64 + 32 * (int64_t)j, df_to_double(z[u]));
              }
            }
          }
          df wv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) wv[u] = ok ? df_mul(t, z[u]) : df{0.f, 0.f};
          df a0 = up16 ? wv[2] : wv[0], a1 = up16 ? wv[3] : wv[1];
          df_acc_add(a0, shfl_xor_df(up16 ? wv[0] : wv[2], 16));
          df_acc_add(a1, shfl_xor_df(up16 ? wv[1] : wv[3], 16));
          df c = up8 ? a1 : a0;
          df_acc_add(c, shfl_xor_df(up8 ? a0 : a1, 8));
          df_acc_add(c, shfl_xor_df(c, 4));
          df_acc_add(c, shfl_xor_df(c, 2));
          df_acc_add(c, shfl_xor_df(c, 1));
          if ((lane & 7) == 0 && j0 + col < r) df_acc_add(bacc[wib][j0 + col], c);
        };
        if (vec && d_other == 2) {
          // two other modes (the common case): the next column group's factor
          // values are fetched while this group is multiplied, stored and
          // reduced, so a lane has two gathers in flight instead of one
          const float* f0 = fhl[0] + 2 * (int64_t)(ok ? __ldg(im) : 0) * r;
          const float* f1 = fhl[1] + 2 * (int64_t)(ok ? __ldg(im + 1) : 0) * r;
          float c0[8], c1[8], n0[8], n1[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) c0[u] = c1[u] = 0.f;
          if (ok) {
            ldg_v8(f0, c0);
            ldg_v8(f1, c1);
          }
          for (int j0 = 0; j0 < r; j0 += 4) {
            const bool more = ok && j0 + 4 < r;
            if (more) {
              ldg_v8(f0 + 2 * (j0 + 4), n0);
              ldg_v8(f1 + 2 * (j0 + 4), n1);
            }
            df z[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              z[u] = ok ? df_mul(df{c0[2 * u], c0[2 * u + 1]}, df{c1[2 * u], c1[2 * u + 1]})
                        : df{0.f, 0.f};
            emit(j0, z);
            if (more) {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                c0[u] = n0[u];
                c1[u] = n1[u];
              }
            }
          }
        } else {
          for (int j0 = 0; j0 < r; j0 += 4) {
            df z[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) z[u] = df{0.f, 0.f};
            if (ok) {
              for (int m = 0; m < d_other; ++m) {
                const int64_t off = (int64_t)__ldg(im + m) * r + j0;
                float h[4], lo[4];
                if (vec) {
                  float v[8];
                  ldg_v8(fhl[m] + 2 * off, v);
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    h[u] = v[2 * u];
                    lo[u] = v[2 * u + 1];
                  }
                } else {
                  const float2* p2 = reinterpret_cast<const float2*>(fhl[m]) + off;
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    const float2 v = j0 + u < r ? __ldg(p2 + u) : make_float2(0.f, 0.f);
                    h[u] = v.x;
                    lo[u] = v.y;
                  }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const df f{h[u], lo[u]};
                  z[u] = m == 0 ? f : df_mul(z[u], f);
                }
              }
            }
            emit(j0, z);
          }
        }
      }
      __syncwarp();
      // the piece's row: directly into B, or a partial row that the last
      // piece of the kernel index adds in piece order
      const int np = pl.seg_count[seg];
      if (np == 1) {
        for (int j = lane; j < r; j += 32)
          B[(int64_t)j * ldb + seg] = df_to_double(df_norm(bacc[wib][j]));
      } else {
        for (int j = lane; j < r; j += 32)
          partial[(int64_t)p * 64 + j] = df_to_double(df_norm(bacc[wib][j]));
        __threadfence();
        __syncwarp();
        unsigned tk = 0;
        if (lane == 0) tk = atomicAdd(&pl.seg_ticket[seg], 1u);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk == (unsigned)(np - 1)) {
          __threadfence();
          const int f = pl.seg_first[seg];
          for (int j = lane; j < r; j += 32) {
            double sacc = 0.0;
            for (int k = 0; k < np; ++k) sacc += __ldcg(&partial[(int64_t)(f + k) * 64 + j]);
            B[(int64_t)j * ldb + seg] = sacc;
          }
          if (lane == 0) pl.seg_ticket[seg] = 0u;
        }
      }
    }
  }
  if (bad) atomicOr(err, bad);  // 1: other-mode index out of range, 2: non-finite value
  if (lane == 0) {  // the last warp out resets the counters
    __threadfence();
    if (atomicAdd(&pl.wctr[1], 1u) == (unsigned)nwarps - 1) {
      pl.wctr[0] = 0u;
      pl.wctr[1] = 0u;
      __threadfence();
    }
  }
}

cudaError_t launch_zhat_mttkrp_fused(const PieceList& pl, int64_t q, const int32_t* perm,
                                     const int32_t* oidx, int d_other, const float* const* fhl,
                                     const int64_t* sizes_dev, int r, const double* vals,
                                     float* zhi, double* z64, double* partial, double* B,
                                     int64_t ldb, int* err, const int* gate, int num_sms,
                                     cudaStream_t st, int w_begin, int w_end) {
  if (w_end < 0) w_end = pl.nwarps;
  if (q == 0 || pl.npieces == 0 || pl.nwarps == 0 || w_end <= w_begin) return cudaSuccess;
  if (d_other < 1 || d_other > 16 || r < 1 || r > 64 || (!zhi && !z64) || !pl.wctr ||
      w_begin < 0 || w_end > pl.nwarps)
    return cudaErrorInvalidValue;
  // one resident wave (4 blocks of 8 warps per SM); the warps draw the ranges
  const int blocks = (int)std::min<int64_t>((w_end - w_begin + 7) / 8, (int64_t)num_sms * 4);
  if (zhi && z64)
    zhat_mttkrp_kernel<true, true><<<blocks, 256, 0, st>>>(pl, q, perm, oidx, d_other, fhl,
                                                           sizes_dev, r, zhi, z64, vals, partial,
                                                           B, ldb, err, gate, w_begin, w_end);
  else if (zhi)
    zhat_mttkrp_kernel<true, false><<<blocks, 256, 0, st>>>(pl, q, perm, oidx, d_other, fhl,
                                                            sizes_dev, r, zhi, z64, vals, partial,
                                                            B, ldb, err, gate, w_begin, w_end);
  else
    zhat_mttkrp_kernel<false, true><<<blocks, 256, 0, st>>>(pl, q, perm, oidx, d_other, fhl,
                                                            sizes_dev, r, zhi, z64, vals, partial,
                                                            B, ldb, err, gate, w_begin, w_end);
  return cudaGetLastError();
}

// Elementwise conversions between the FP64 Zhat and its interleaved FP32 pair.
__global__ void zhat_split_kernel(const double* __restrict__ z64, int64_t total, int r,
                                  float* __restrict__ zhl) {
  const int64_t per = 32 * (int64_t)r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = t / per, in = t - tile * per;
    const df d = df_from_double(z64[t]);
    zhl[tile * 2 * per + in] = d.hi;
    zhl[tile * 2 * per + per + in] = d.lo;
  }
}

__global__ void zhat_join_kernel(const float* __restrict__ zhl, int64_t total, int r,
                                 double* __restrict__ z64) {
  const int64_t per = 32 * (int64_t)r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = t / per, in = t - tile * per;
    z64[t] = (double)zhl[tile * 2 * per + in] + (double)zhl[tile * 2 * per + per + in];
  }
}

cudaError_t launch_zhat_split(const double* z64, int64_t q, int r, float* zhl, cudaStream_t st) {
  const int64_t total = zhat_elems(q, r);
  if (total == 0) return cudaSuccess;
  int64_t b = (total + 255) / 256;
  if (b > 8192) b = 8192;
  zhat_split_kernel<<<(int)b, 256, 0, st>>>(z64, total, r, zhl);
  return cudaGetLastError();
}

cudaError_t launch_zhat_join(const float* zhl, int64_t q, int r, double* z64, cudaStream_t st) {
  const int64_t total = zhat_elems(q, r);
  if (total == 0) return cudaSuccess;
  int64_t b = (total + 255) / 256;
  if (b > 8192) b = 8192;
  zhat_join_kernel<<<(int)b, 256, 0, st>>>(zhl, total, r, z64);
  return cudaGetLastError();
}

cudaError_t launch_gds_f32(const PieceList& pl, const float* zhi, int r, const float* Xh,
                           int64_t xld, float* partial, float* Y, int64_t yld,
                           const DevScalars* skip, cudaStream_t st) {
  return gds_by_rank<GDS_F32>(pl, zhi, nullptr, nullptr, r, Xh, xld, partial, Y, yld, skip, st);
}
cudaError_t launch_gds_f64(const PieceList& pl, const double* z64, int r, const double* Xh,
                           int64_t xld, double* partial, double* Y, int64_t yld,
                           const DevScalars* skip, cudaStream_t st) {
  return gds_by_rank<GDS_F64>(pl, nullptr, nullptr, z64, r, Xh, xld, partial, Y, yld, skip, st);
}
cudaError_t launch_gds_df(const PieceList& pl, const float* zhi, const float* zlo, int r,
                          const double* Xh, int64_t xld, double* partial, double* Y, int64_t yld,
                          const DevScalars* skip, cudaStream_t st) {
  return gds_by_rank<GDS_DF>(pl, zhi, zlo, nullptr, r, Xh, xld, partial, Y, yld, skip, st);
}

}  // namespace cphifi
