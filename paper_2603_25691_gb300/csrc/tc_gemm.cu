// Tensor-core (tcgen05) skinny products for the mixed operator: the two n x n
// products of an iteration, X̂ = U_K (D_K P̄) and U_K' Ŷ1 (§4.4.1 "K X" and
// "K Yhat1" in the eigenbasis), with TF32 or BF16 operands and FP32
// accumulation in tensor memory.
//
// C_split(i, j) = sum_{k in split} A(i, k) B(k, j) for a 128-row tile of A per
// block and a range of k per split.  Both operands are K-major:
//   A: rows of A are contiguous in k (U_K' is U_K column-major; U_K itself
//      uses a transposed copy), tensor map dims {K, M};
//   B: the n x ncols column-major vector block, tensor map dims {K, N}; rows
//      N >= ncols of the box are zero-filled by the TMA unit.
// One block = 4 warps.  Warp 0 (one lane) streams 128-byte-wide k slabs of A
// and B into a ring of shared-memory stages with TMA (128-byte swizzle);
// warp 1 (one lane) issues tcgen05.mma (M = 128, N = NP, 32 bytes of k per
// instruction) into a TMEM accumulator and releases each stage with
// tcgen05.commit; after the last slab all four warps read their 32 TMEM lanes
// (tcgen05.ld) and store FP32 partial sums.  Every mbarrier wait is bounded:
// on expiry the kernel records an error code and returns after freeing its
// TMEM (no trap, no endless spin).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"
#include "tc_util.cuh"

namespace cphifi {

namespace {

constexpr int kTcStages = 6;
constexpr int kTcBlock = 128;

}  // namespace

using namespace tcu;

// SPLIT3 (TF32 only): the operands come as hi + lo pairs of TF32 values
// (tensor maps tmAl, tmBl for the lo parts) and each k step accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi: the 3-term split product, accurate to
// about 2^-21 instead of TF32's 2^-11.
template <typename T, int NP, bool SPLIT3>
__global__ void __launch_bounds__(kTcBlock, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmAl, const __grid_constant__ CUtensorMap tmBl,
               float* __restrict__ C, int64_t ldc, int64_t split_stride, int n, int ncols,
               int kchunk, const DevScalars* skip, int* err) {
  if (dev_skip(skip)) return;
  constexpr int BK = 128 / (int)sizeof(T);            // k per 128-byte slab
  constexpr int A_BYTES = 128 * 128;                  // 128 rows x 128 bytes
  constexpr int B_BYTES = NP * 128;
  constexpr int STAGE = (A_BYTES + B_BYTES) * (SPLIT3 ? 2 : 1);
  constexpr int kStages = SPLIT3 ? 4 : kTcStages;
  constexpr uint32_t TMEM_COLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full_bar[kTcStages], empty_bar[kTcStages], done_bar;  // kStages used
  __shared__ uint32_t tmem_slot;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  const int kbeg = blockIdx.y * kchunk;
  const int kend = min(n, kbeg + kchunk);
  const int nslab = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (nslab > 0) {
    if (warp == 0 && lane == 0) {
      // producer: TMA ring
      for (int c = 0; c < nslab; ++c) {
        const int s = c % kStages;
        const uint32_t ph = (uint32_t)(c / kStages) & 1u;
        if (c >= kStages && !mbar_wait(&empty_bar[s], ph ^ 1u, err, 1)) break;
        uint8_t* st = smem + s * STAGE;
        mbar_expect_tx(&full_bar[s], STAGE);
        tma_load_2d(st, &tmA, kbeg + c * BK, m0, &full_bar[s]);
        tma_load_2d(st + A_BYTES, &tmB, kbeg + c * BK, 0, &full_bar[s]);
        if (SPLIT3) {
          tma_load_2d(st + A_BYTES + B_BYTES, &tmAl, kbeg + c * BK, m0, &full_bar[s]);
          tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tmBl, kbeg + c * BK, 0, &full_bar[s]);
        }
      }
    } else if (warp == 1 && lane == 0) {
      // MMA issuer
      const uint32_t id = idesc<T>(NP);
      for (int c = 0; c < nslab; ++c) {
        const int s = c % kStages;
        const uint32_t ph = (uint32_t)(c / kStages) & 1u;
        if (!mbar_wait(&full_bar[s], ph, err, 2)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint8_t* st = smem + s * STAGE;
        const uint8_t* ah = st;
        const uint8_t* bh = st + A_BYTES;
#pragma unroll
        for (int kk = 0; kk < 128 / 32; ++kk) {
          mma<T>(tmem, sdesc(ah + kk * 32), sdesc(bh + kk * 32), id, (c > 0 || kk > 0) ? 1u : 0u);
          if (SPLIT3) {
            const uint8_t* al = st + A_BYTES + B_BYTES;
            const uint8_t* bl = st + 2 * A_BYTES + B_BYTES;
            mma<T>(tmem, sdesc(ah + kk * 32), sdesc(bl + kk * 32), id, 1u);
            mma<T>(tmem, sdesc(al + kk * 32), sdesc(bh + kk * 32), id, 1u);
          }
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&done_bar);
    }
    __syncwarp();
    // epilogue: TMEM lanes 32w..32w+31 hold rows m0 + 32w + lane
    const bool ok = mbar_wait(&done_bar, 0, err, 4);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    float* Cs = C + (int64_t)blockIdx.y * split_stride;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
          "%10, %11, %12, %13, %14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
            "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
            "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (ok && row < n) {
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (c0 + t < ncols) Cs[(int64_t)(c0 + t) * ldc + row] = __uint_as_float(v[t]);
      }
    }
  } else {
    const int row = m0 + warp * 32 + lane;
    float* Cs = C + (int64_t)blockIdx.y * split_stride;
    if (row < n)
      for (int j = 0; j < ncols; ++j) Cs[(int64_t)j * ldc + row] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// ------------------------------------------------------------------ host ---
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  }
  return fn;
}
}  // namespace

// The operand copies use a leading dimension padded to a multiple of 8
// elements, so TMA's 16-byte row strides hold for every n.
bool tc_available(int n) { return encode_fn() != nullptr && n >= 1; }

cudaError_t tc_make_map(CUtensorMap* map, const void* base, bool bf16, uint64_t inner,
                        uint64_t outer, uint64_t row_stride_bytes, uint32_t box_outer) {
  EncodeFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_stride_bytes};
  const cuuint32_t box[2] = {bf16 ? 64u : 32u, box_outer};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_pad_cols(int ncols) { return ncols <= 16 ? 16 : (ncols <= 32 ? 32 : (ncols <= 48 ? 48 : 64)); }

int tc_pick_split(int n, int num_sms) {
  const int mt = (n + 127) / 128;
  int s = num_sms / mt;  // one wave of one block per SM (the block holds ~140 KB of stages)
  const int slabs = (n + 31) / 32;
  if (s > slabs) s = slabs;
  if (s > 64) s = 64;
  return s < 1 ? 1 : s;
}

template <typename T, int NP, bool SPLIT3>
static cudaError_t tc_launch(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mal,
                             const CUtensorMap& mbl, float* C, int64_t ldc, int64_t split_stride,
                             int n, int ncols, int nsplit, const DevScalars* skip, int* err,
                             cudaStream_t st) {
  constexpr int STAGE = (128 * 128 + NP * 128) * (SPLIT3 ? 2 : 1);
  constexpr int kStages = SPLIT3 ? 4 : kTcStages;
  const size_t smem = (size_t)kStages * STAGE + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<T, NP, SPLIT3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  constexpr int BK = 128 / (int)sizeof(T);
  int kchunk = (n + nsplit - 1) / nsplit;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const dim3 grid((n + 127) / 128, nsplit);
  tc_gemm_kernel<T, NP, SPLIT3><<<grid, kTcBlock, smem, st>>>(ma, mb, mal, mbl, C, ldc,
                                                              split_stride, n, ncols, kchunk,
                                                              skip, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(bool bf16, const CUtensorMap& ma, const CUtensorMap& mb,
                           const CUtensorMap* mal, const CUtensorMap* mbl, float* C, int64_t ldc,
                           int64_t split_stride, int n, int ncols, int nsplit,
                           const DevScalars* skip, int* err, cudaStream_t st) {
  const int np = tc_pad_cols(ncols);
  const bool split3 = !bf16 && mal && mbl;
  const CUtensorMap& al = split3 ? *mal : ma;
  const CUtensorMap& bl = split3 ? *mbl : mb;
#define CPHIFI_TC(NPV)                                                                        \
  if (bf16)                                                                                   \
    return tc_launch<__nv_bfloat16, NPV, false>(ma, mb, al, bl, C, ldc, split_stride, n,      \
                                                ncols, nsplit, skip, err, st);                \
  if (split3)                                                                                 \
    return tc_launch<float, NPV, true>(ma, mb, al, bl, C, ldc, split_stride, n, ncols, nsplit, \
                                       skip, err, st);                                        \
  return tc_launch<float, NPV, false>(ma, mb, al, bl, C, ldc, split_stride, n, ncols, nsplit,  \
                                      skip, err, st)
  if (np == 16) { CPHIFI_TC(16); }
  if (np == 32) { CPHIFI_TC(32); }
  if (np == 48) { CPHIFI_TC(48); }
  CPHIFI_TC(64);
#undef CPHIFI_TC
}

// Operand preparation for the tensor-core products.
// U_K (FP64, column-major) -> FP32 or BF16 copy, transposed (row-major U_K,
// the K-major A operand of U_K X) or not (the K-major A of U_K' X).
template <typename T>
__global__ void uk_copy_kernel(const double* __restrict__ U, int n, int64_t ldo, bool transpose,
                               T* __restrict__ out) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int i = bx + threadIdx.x, j = by + k;  // read U(i, j) at i + n j (coalesced in i)
    tile[k][threadIdx.x] = (i < n && j < n) ? U[(int64_t)j * n + i] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    if (transpose) {
      const int i = bx + k, j = by + threadIdx.x;  // write out[i * n + j] = U(i, j)
      if (i < n && j < n) out[(int64_t)i * ldo + j] = (T)tile[threadIdx.x][k];
    } else {
      const int i = bx + threadIdx.x, j = by + k;  // out[i + n j] = U(i, j)
      if (i < n && j < n) out[(int64_t)j * ldo + i] = (T)tile[k][threadIdx.x];
    }
  }
}

template <typename T>
cudaError_t launch_uk_copy(const double* U, int n, int64_t ldo, bool transpose, T* out,
                           cudaStream_t st) {
  const dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  uk_copy_kernel<T><<<grid, block, 0, st>>>(U, n, ldo, transpose, out);
  return cudaGetLastError();
}
template cudaError_t launch_uk_copy<float>(const double*, int, int64_t, bool, float*, cudaStream_t);
template cudaError_t launch_uk_copy<__nv_bfloat16>(const double*, int, int64_t, bool,
                                                   __nv_bfloat16*, cudaStream_t);

// TF32 split: hi = x with the 13 low significand bits cleared (a TF32 value),
// lo = x - hi (exact in FP32; its TF32 rounding loses ~2^-21 of x).
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

// hi/lo TF32 split of U_K copies, in place for hi (a) and into lo.
__global__ void tf32_split_kernel(float* __restrict__ a, float* __restrict__ lo, int64_t total) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    float h, l;
    tf32_split(a[t], h, l);
    a[t] = h;
    lo[t] = l;
  }
}

cudaError_t launch_tf32_split(const float* src, float* hi, float* lo, int64_t total,
                              cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  if (src != hi) {
    cudaError_t e = cudaMemcpyAsync(hi, src, total * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  int64_t b = (total + 255) / 256;
  if (b > 4096) b = 4096;
  tf32_split_kernel<<<(int)b, 256, 0, st>>>(hi, lo, total);
  return cudaGetLastError();
}

// Strided hi/lo TF32 split of an n x r block (ld ldx) into hi/lo (ld ldo).
__global__ void tf32_split_block_kernel(const float* __restrict__ x, int64_t ldx, int64_t rows,
                                        int64_t total, float* __restrict__ hi,
                                        float* __restrict__ lo, int64_t ldo,
                                        const DevScalars* skip) {
  if (dev_skip(skip)) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, j = t / rows;
    float h, l;
    tf32_split(x[j * ldx + i], h, l);
    hi[j * ldo + i] = h;
    lo[j * ldo + i] = l;
  }
}

cudaError_t launch_tf32_split_block(const float* x, int64_t ldx, int64_t rows, int64_t total,
                                    float* hi, float* lo, int64_t ldo, const DevScalars* skip,
                                    cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  int64_t b = (total + 255) / 256;
  if (b > 2048) b = 2048;
  tf32_split_block_kernel<<<(int)b, 256, 0, st>>>(x, ldx, rows, total, hi, lo, ldo, skip);
  return cudaGetLastError();
}

// out = T(scale[i] * X(i, j)) for an n x r column-major block (scale may be
// NULL): the B operand of the tensor-core products.
template <typename TS, typename T>
__global__ void scale_to_kernel(const TS* __restrict__ X, const double* __restrict__ scale,
                                int64_t rows, int64_t total, T* __restrict__ out, int64_t ldo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % rows, j = t / rows;
    const double v = scale ? scale[i] * (double)X[t] : (double)X[t];
    out[j * ldo + i] = (T)v;
  }
}

template <typename TS, typename T>
cudaError_t launch_scale_to(const TS* X, const double* scale, int64_t rows, int64_t total, T* out,
                            int64_t ldo, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  int64_t b = (total + 255) / 256;
  if (b > 2048) b = 2048;
  scale_to_kernel<TS, T><<<(int)b, 256, 0, st>>>(X, scale, rows, total, out, ldo);
  return cudaGetLastError();
}
template cudaError_t launch_scale_to<double, float>(const double*, const double*, int64_t, int64_t,
                                                    float*, int64_t, cudaStream_t);
template cudaError_t launch_scale_to<double, __nv_bfloat16>(const double*, const double*, int64_t,
                                                            int64_t, __nv_bfloat16*, int64_t,
                                                            cudaStream_t);
template cudaError_t launch_scale_to<float, __nv_bfloat16>(const float*, const double*, int64_t,
                                                           int64_t, __nv_bfloat16*, int64_t,
                                                           cudaStream_t);

}  // namespace cphifi
