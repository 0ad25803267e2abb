// Skinny dense products with the kernel eigenbasis (§4.4.1 "K X" and
// "K Yhat1", §4.4.2 "U_K' X", "U_K S"): C = op(A) diag(s) B where A is the
// n x n eigenvector matrix U_K, B is n x r (r <= 64) and s an optional
// per-row scale of B (the eigenvalues D_K).  op(A)(i,k) is read as
// A[k*lda + i] when a_trans is true (A column-major, i.e. U_K itself) and as
// A[i*lda + k] otherwise (U_K').  The k-range is split so that the grid
// covers every SM; partial products are combined (and the elementwise tail
// of the operator applied) by the combine kernel in cg.cu.
//
// SIMT FP64/FP32 version: 256 threads, a 128 x r tile of C per block,
// 32-wide (FP32) or 16-wide (FP64) k slabs staged through shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "launch.h"

namespace cphifi {

template <typename TA, typename TC, bool ATRANS, bool SCALEB>
__global__ void __launch_bounds__(256)
gemm_skinny_kernel(const TA* __restrict__ A, int64_t lda, const double* __restrict__ sk,
                   const TC* __restrict__ B, int64_t ldb, TC* __restrict__ C, int64_t ldc,
                   int64_t split_stride, int n, int ncols, int kchunk, const DevScalars* skip) {
  if (dev_skip(skip)) return;
  // 16-wide k slabs in FP64 keep the static shared memory under 48 KB.
  constexpr int BM = 128, BK = sizeof(TC) == 8 ? 16 : 32, TM = BM / 32, TNMAX = 8;
  __shared__ TC As[BK][BM + 1];
  __shared__ TC Bs[BK][64];
  const int tid = threadIdx.x;
  const int ty = tid & 31;       // row group: rows ty, ty+32, ty+64, ty+96
  const int tx = tid >> 5;       // column group
  const int tn = (ncols + 7) / 8;  // columns per thread (<= 8)
  const int i0 = blockIdx.x * BM;
  const int kbeg = blockIdx.y * kchunk;
  const int kend = min(n, kbeg + kchunk);
  TC acc[TM][TNMAX];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TNMAX; ++b) acc[a][b] = TC(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    if (ATRANS) {
      for (int idx = tid; idx < BM * BK; idx += 256) {
        const int ii = idx % BM, kk = idx / BM;
        const int i = i0 + ii, k = k0 + kk;
        As[kk][ii] = (i < n && k < kend) ? TC(A[(int64_t)k * lda + i]) : TC(0);
      }
    } else {
      for (int idx = tid; idx < BM * BK; idx += 256) {
        const int kk = idx % BK, ii = idx / BK;
        const int i = i0 + ii, k = k0 + kk;
        As[kk][ii] = (i < n && k < kend) ? TC(A[(int64_t)i * lda + k]) : TC(0);
      }
    }
    for (int idx = tid; idx < BK * 64; idx += 256) {
      const int kk = idx % BK, j = idx / BK;
      const int k = k0 + kk;
      TC v = TC(0);
      if (k < kend && j < ncols) {
        v = B[(int64_t)j * ldb + k];
        if (SCALEB) v = TC(double(v) * sk[k]);
      }
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      TC a[TM], b[TNMAX];
#pragma unroll
      for (int m = 0; m < TM; ++m) a[m] = As[kk][ty + 32 * m];
#pragma unroll
      for (int c = 0; c < TNMAX; ++c) b[c] = c < tn ? Bs[kk][tx * tn + c] : TC(0);
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int c = 0; c < TNMAX; ++c) acc[m][c] = fma(a[m], b[c], acc[m][c]);
    }
    __syncthreads();
  }
  TC* Cs = C + (int64_t)blockIdx.y * split_stride;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int i = i0 + ty + 32 * m;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < TNMAX; ++c) {
      const int j = tx * tn + c;
      if (c < tn && j < ncols) Cs[(int64_t)j * ldc + i] = acc[m][c];
    }
  }
}

// FP32 version with a larger register tile: 256 rows per block, each thread
// 8 rows (ty + 32 m) x tn columns, so a k step costs 8 + tn shared loads for
// 8 tn multiply-adds; the next slab of A and B is fetched into registers
// while the current one is multiplied (one __syncthreads per slab).
constexpr int kF32BM = 256, kF32BK = 16;

template <bool ATRANS, bool SCALEB, int TNMAX>
__global__ void __launch_bounds__(256, 2)
gemm_f32_kernel(const float* __restrict__ A, int64_t lda, const double* __restrict__ sk,
                const float* __restrict__ B, int64_t ldb, float* __restrict__ C, int64_t ldc,
                int64_t split_stride, int n, int ncols, int kchunk, const DevScalars* skip) {
  if (dev_skip(skip)) return;
  constexpr int BM = kF32BM, BK = kF32BK, TM = BM / 32;
  constexpr int AL = BM * BK / 256;  // A values each thread stages per slab (16)
  constexpr int BL = BK * 64 / 256;  // B values each thread stages per slab (4)
  // A tile rows: thread ty owns rows 4ty..4ty+3 and 128+4ty..128+4ty+3 (two
  // 128-bit shared loads per k); B: warp tx's TNMAX columns at [8 tx, 8 tx +
  // TNMAX) of a 64-float row (two 128-bit broadcast loads per k).
  static_assert(BM == 256 && TNMAX <= 8, "register tile of 8 rows x 8 columns at most");
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][64];
  const int tid = threadIdx.x;
  const int ty = tid & 31, tx = tid >> 5;
  const int i0 = blockIdx.x * BM;  // columns tx*TNMAX .. +TNMAX-1 (< 64)
  const int kbeg = blockIdx.y * kchunk;
  const int kend = min(n, kbeg + kchunk);
  float acc[TM][TNMAX];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TNMAX; ++b) acc[a][b] = 0.f;
  float ra[AL], rb[BL];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + 256 * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      const int i = i0 + ii, k = k0 + kk;
      ra[u] = (i < n && k < kend)
                  ? __ldg(ATRANS ? A + (int64_t)k * lda + i : A + (int64_t)i * lda + k)
                  : 0.f;
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + 256 * u;
      const int kk = idx % BK, j = idx / BK;
      const int k = k0 + kk;
      float v = 0.f;
      if (k < kend && j < ncols) {
        v = __ldg(B + (int64_t)j * ldb + k);
        if (SCALEB) v = (float)((double)v * sk[k]);
      }
      rb[u] = v;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + 256 * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      As[buf][kk][ii] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + 256 * u;
      const int j = idx / BK;
      if (j < 8 * TNMAX) Bs[buf][idx % BK][(j / TNMAX) * 8 + j % TNMAX] = rb[u];
    }
  };
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) fetch(k0 + BK);  // in flight during the multiply below
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][128 + 4 * ty]);
      const float a[TM] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][8 * tx]);
      float4 b1 = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (TNMAX > 4) b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][8 * tx + 4]);
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int c = 0; c < TNMAX; ++c) acc[m][c] = fmaf(a[m], bv[c], acc[m][c]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* Cs = C + (int64_t)blockIdx.y * split_stride;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int i = i0 + (m < 4 ? 4 * ty + m : 128 + 4 * ty + m - 4);
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < TNMAX; ++c) {
      const int j = tx * TNMAX + c;
      if (j < ncols) Cs[(int64_t)j * ldc + i] = acc[m][c];
    }
  }
}

// Split of the k range: the grid is (ceil(n/128) row tiles) x nsplit blocks;
// pick nsplit so that the blocks fill whole waves of the resident slots
// (SMs x blocks per SM) as evenly as possible -- a grid of 1.04 waves runs
// as long as two.
template <typename TA, typename TC>
int gemm_pick_split(int n, int num_sms) {
  constexpr bool f32 = sizeof(TC) == 4;
  int occ = 1;
  if (f32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gemm_f32_kernel<true, true, 5>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gemm_skinny_kernel<TA, TC, true, true>, 256, 0);
  if (occ < 1) occ = 1;
  const int64_t slots = (int64_t)num_sms * occ;
  const int bm = f32 ? kF32BM : 128;
  const int mt = (n + bm - 1) / bm;
  int smax = (n + 31) / 32;
  if (smax > 32) smax = 32;
  int best = 1;
  double best_eff = -1.0;
  for (int s = 1; s <= smax; ++s) {
    const int64_t ctas = (int64_t)mt * s;
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots);
    if (eff > best_eff + 0.02) { best_eff = eff; best = s; }
  }
  return best;
}

template int gemm_pick_split<double, double>(int, int);
template int gemm_pick_split<float, float>(int, int);

template <typename TA, typename TC>
cudaError_t launch_gemm_skinny(const TA* A, int64_t lda, bool a_trans, const double* scale_k,
                               const TC* B, int64_t ldb, TC* C, int64_t ldc,
                               int64_t split_stride, int n, int ncols, int nsplit,
                               const DevScalars* skip, cudaStream_t st) {
  if (n == 0 || ncols == 0) return cudaSuccess;
  if (ncols > 64) return cudaErrorInvalidValue;
  int kchunk = (n + nsplit - 1) / nsplit;
  kchunk = (kchunk + 31) / 32 * 32;
  if constexpr (sizeof(TA) == 4 && sizeof(TC) == 4) {
    const dim3 g((n + kF32BM - 1) / kF32BM, nsplit);
    const float* Af = reinterpret_cast<const float*>(A);
    const float* Bf = reinterpret_cast<const float*>(B);
    float* Cf = reinterpret_cast<float*>(C);
    const int tn = (ncols + 7) / 8;
#define CPHIFI_F32(TNV)                                                                           \
  do {                                                                                            \
    if (a_trans) {                                                                                \
      if (scale_k) gemm_f32_kernel<true, true, TNV><<<g, 256, 0, st>>>(Af, lda, scale_k, Bf, ldb, Cf, ldc, split_stride, n, ncols, kchunk, skip);   \
      else gemm_f32_kernel<true, false, TNV><<<g, 256, 0, st>>>(Af, lda, scale_k, Bf, ldb, Cf, ldc, split_stride, n, ncols, kchunk, skip);         \
    } else {                                                                                      \
      if (scale_k) gemm_f32_kernel<false, true, TNV><<<g, 256, 0, st>>>(Af, lda, scale_k, Bf, ldb, Cf, ldc, split_stride, n, ncols, kchunk, skip);  \
      else gemm_f32_kernel<false, false, TNV><<<g, 256, 0, st>>>(Af, lda, scale_k, Bf, ldb, Cf, ldc, split_stride, n, ncols, kchunk, skip);        \
    }                                                                                             \
  } while (0)
    if (tn <= 1) CPHIFI_F32(1);
    else if (tn <= 2) CPHIFI_F32(2);
    else if (tn <= 3) CPHIFI_F32(3);
    else if (tn <= 4) CPHIFI_F32(4);
    else if (tn <= 5) CPHIFI_F32(5);
    else if (tn <= 6) CPHIFI_F32(6);
    else CPHIFI_F32(8);
#undef CPHIFI_F32
    return cudaGetLastError();
  }
  const dim3 grid((n + 127) / 128, nsplit);
  if (a_trans) {
    if (scale_k)
      gemm_skinny_kernel<TA, TC, true, true><<<grid, 256, 0, st>>>(A, lda, scale_k, B, ldb, C, ldc, split_stride, n, ncols, kchunk, skip);
    else
      gemm_skinny_kernel<TA, TC, true, false><<<grid, 256, 0, st>>>(A, lda, scale_k, B, ldb, C, ldc, split_stride, n, ncols, kchunk, skip);
  } else {
    if (scale_k)
      gemm_skinny_kernel<TA, TC, false, true><<<grid, 256, 0, st>>>(A, lda, scale_k, B, ldb, C, ldc, split_stride, n, ncols, kchunk, skip);
    else
      gemm_skinny_kernel<TA, TC, false, false><<<grid, 256, 0, st>>>(A, lda, scale_k, B, ldb, C, ldc, split_stride, n, ncols, kchunk, skip);
  }
  return cudaGetLastError();
}

// Double-float version (FP64-accurate products of the mixed solve: the
// right-hand side, the true residual, W = U_K Wbar).  A and B arrive as hi/lo
// FP32 pairs (A = U_K split once per kernel, B split per call with the
// optional row scale folded in); every multiply-add is an exact TwoProd and a
// TwoSum-compensated accumulation (df.cuh), the partial products are written
// as FP64.  FP32 units only: GB300 runs them ~60x faster than FP64 FMA.
// TNMAX = columns per thread (ncols <= 8 TNMAX), a compile-time bound that
// keeps the accumulator tile in registers without padding to 64 columns.
template <bool ATRANS, int TNMAX>
__global__ void __launch_bounds__(256)
gemm_df_kernel(const float* __restrict__ Ahi, const float* __restrict__ Alo, int64_t lda,
               const float* __restrict__ Bhi, const float* __restrict__ Blo, int64_t ldb,
               double* __restrict__ C, int64_t ldc, int64_t split_stride, int n, int ncols,
               int kchunk, const DevScalars* skip) {
  if (dev_skip(skip)) return;
  constexpr int BM = 128, BK = 16, TM = BM / 32;
  constexpr int AL = BM * BK / 256, BL = BK * 64 / 256;  // staged values per thread
  __shared__ float Ash[BK][BM + 1], Asl[BK][BM + 1];
  __shared__ float Bsh[BK][64], Bsl[BK][64];
  const int tid = threadIdx.x;
  const int ty = tid & 31, tx = tid >> 5;
  const int i0 = blockIdx.x * BM;  // columns tx*TNMAX .. +TNMAX-1 (< 64)
  const int kbeg = blockIdx.y * kchunk;
  const int kend = min(n, kbeg + kchunk);
  df acc[TM][TNMAX];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TNMAX; ++b) acc[a][b] = df{0.f, 0.f};
  // the next slab is fetched into registers while the current one is used
  float rah[AL], ral[AL], rbh[BL], rbl[BL];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + 256 * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      const int i = i0 + ii, k = k0 + kk;
      float h = 0.f, l = 0.f;
      if (i < n && k < kend) {
        const int64_t off = ATRANS ? (int64_t)k * lda + i : (int64_t)i * lda + k;
        h = __ldg(Ahi + off);
        l = __ldg(Alo + off);
      }
      rah[u] = h;
      ral[u] = l;
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + 256 * u;
      const int kk = idx % BK, j = idx / BK;
      const int k = k0 + kk;
      float h = 0.f, l = 0.f;
      if (k < kend && j < ncols) {
        h = __ldg(Bhi + (int64_t)j * ldb + k);
        l = __ldg(Blo + (int64_t)j * ldb + k);
      }
      rbh[u] = h;
      rbl[u] = l;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + 256 * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      Ash[kk][ii] = rah[u];
      Asl[kk][ii] = ral[u];
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + 256 * u;
      Bsh[idx % BK][idx / BK] = rbh[u];
      Bsl[idx % BK][idx / BK] = rbl[u];
    }
  };
  if (kbeg < kend) {
    fetch(kbeg);
    stash();
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) fetch(k0 + BK);
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      df a[TM], b[TNMAX];
#pragma unroll
      for (int m = 0; m < TM; ++m) a[m] = df{Ash[kk][ty + 32 * m], Asl[kk][ty + 32 * m]};
#pragma unroll
      for (int c = 0; c < TNMAX; ++c)
        b[c] = df{Bsh[kk][tx * TNMAX + c], Bsl[kk][tx * TNMAX + c]};
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int c = 0; c < TNMAX; ++c)
          df_acc_prod(acc[m][c], a[m], b[c]);
    }
    __syncthreads();
    if (more) stash();
    __syncthreads();
  }
  double* Cs = C + (int64_t)blockIdx.y * split_stride;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int i = i0 + ty + 32 * m;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < TNMAX; ++c) {
      const int j = tx * TNMAX + c;
      if (j < ncols) Cs[(int64_t)j * ldc + i] = df_to_double(df_norm(acc[m][c]));
    }
  }
}

int gemm_df_pick_split(int n, int num_sms) {
  int occ = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gemm_df_kernel<true, 5>, 256, 0);
  if (occ < 1) occ = 1;
  const int64_t slots = (int64_t)num_sms * occ;
  const int mt = (n + 127) / 128;
  int smax = (n + 15) / 16;
  if (smax > 32) smax = 32;
  int best = 1;
  double best_eff = -1.0;
  for (int s = 1; s <= smax; ++s) {
    const int64_t ctas = (int64_t)mt * s;
    const int64_t waves = (ctas + slots - 1) / slots;
    const double eff = (double)ctas / (double)(waves * slots);
    if (eff > best_eff + 0.02) { best_eff = eff; best = s; }
  }
  return best;
}

cudaError_t launch_gemm_df(const float* Ahi, const float* Alo, int64_t lda, bool a_trans,
                           const float* Bhi, const float* Blo, int64_t ldb, double* C, int64_t ldc,
                           int64_t split_stride, int n, int ncols, int nsplit,
                           const DevScalars* skip, cudaStream_t st) {
  if (n == 0 || ncols == 0) return cudaSuccess;
  if (ncols > 64) return cudaErrorInvalidValue;
  int kchunk = (n + nsplit - 1) / nsplit;
  kchunk = (kchunk + 15) / 16 * 16;
  const dim3 grid((n + 127) / 128, nsplit);
  const int tn = (ncols + 7) / 8;
#define CPHIFI_GDF(TNV)                                                                        \
  do {                                                                                         \
    if (a_trans)                                                                               \
      gemm_df_kernel<true, TNV><<<grid, 256, 0, st>>>(Ahi, Alo, lda, Bhi, Blo, ldb, C, ldc,    \
                                                      split_stride, n, ncols, kchunk, skip);   \
    else                                                                                       \
      gemm_df_kernel<false, TNV><<<grid, 256, 0, st>>>(Ahi, Alo, lda, Bhi, Blo, ldb, C, ldc,   \
                                                       split_stride, n, ncols, kchunk, skip);  \
  } while (0)
  if (tn <= 1) CPHIFI_GDF(1);
  else if (tn <= 2) CPHIFI_GDF(2);
  else if (tn <= 3) CPHIFI_GDF(3);
  else if (tn <= 4) CPHIFI_GDF(4);
  else if (tn <= 5) CPHIFI_GDF(5);
  else if (tn <= 6) CPHIFI_GDF(6);
  else CPHIFI_GDF(8);
#undef CPHIFI_GDF
  return cudaGetLastError();
}

// hi + lo = scale[i] * X(i, j) (scale may be NULL), the double-float operand
// of gemm_df_kernel.
__global__ void split_df_kernel(const double* __restrict__ X, const double* __restrict__ scale,
                                int64_t rows, int64_t total, float* __restrict__ hi,
                                float* __restrict__ lo) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double v = scale ? scale[t % rows] * X[t] : X[t];
    const df d = df_from_double(v);
    hi[t] = d.hi;
    lo[t] = d.lo;
  }
}

cudaError_t launch_split_df(const double* X, const double* scale, int64_t rows, int64_t total,
                            float* hi, float* lo, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  int64_t b = (total + 255) / 256;
  if (b > 4096) b = 4096;
  split_df_kernel<<<(int)b, 256, 0, st>>>(X, scale, rows, total, hi, lo);
  return cudaGetLastError();
}

__global__ void split_rows_df_kernel(const double* __restrict__ X, int64_t rows, int cols,
                                     float2* __restrict__ hl) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols;
    const int j = (int)(t % cols);
    const df d = df_from_double(X[i + rows * j]);
    hl[t] = make_float2(d.hi, d.lo);
  }
}

cudaError_t launch_split_rows_df(const double* X, int64_t rows, int cols, float* hl,
                                 cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total == 0) return cudaSuccess;
  int64_t b = (total + 255) / 256;
  if (b > 4096) b = 4096;
  split_rows_df_kernel<<<(int)b, 256, 0, st>>>(X, rows, cols, reinterpret_cast<float2*>(hl));
  return cudaGetLastError();
}

template cudaError_t launch_gemm_skinny<double, double>(const double*, int64_t, bool, const double*,
                                                        const double*, int64_t, double*, int64_t,
                                                        int64_t, int, int, int, const DevScalars*,
                                                        cudaStream_t);
template cudaError_t launch_gemm_skinny<float, float>(const float*, int64_t, bool, const double*,
                                                      const float*, int64_t, float*, int64_t,
                                                      int64_t, int, int, int, const DevScalars*,
                                                      cudaStream_t);

}  // namespace cphifi
