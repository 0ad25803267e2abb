// Per-index Gram blocks of the matrix-free product (§4.4.1).
//
// Row i of Yhat1 collects only the observations with i_l = i, and each adds
// (Xhat(i,:).Zhat(l,:)) Zhat(l,:) = (Zhat(l,:)'Zhat(l,:)) Xhat(i,:)' (Eqs. vl
// and yhat1), so
//     Yhat1(i,:)' = C_i Xhat(i,:)',   C_i = sum_{l: i_l = i} Zhat(l,:)'Zhat(l,:),
// the r x r diagonal blocks of H in F'F = (I (x) K) H (I (x) K).  Once the
// n r^2 values of the blocks are formed (one pass over Zhat, q r^2 / 2
// multiply-adds), every later product reads n r^2 values instead of the q r
// of Zhat: at q / n = 6250 observations per index and r = 40 that is 1.6k
// instead of 250k values per index.
//
// gram_build_f32_tiled_kernel (FP32 blocks, r <= 48) is described where it is
// defined.  gram_build_kernel (FP64-accurate blocks; FP32 for 48 < r <= 64):
// a segmented SYRK over the sorted observations.  The
// observations are cut into pieces (one kernel index, at most L of its
// observations); a block takes a piece, stages each 32-observation tile of
// Zhat in shared memory (observation-major) and accumulates its tile of the
// upper triangle of C_i: 16 x 16 threads, thread (ty, tx) owning rows
// ty T .. ty T + T - 1 and columns tx T .. (T = RP / 16), the threads below
// the diagonal idle.  An index covered by one piece writes C_i directly;
// otherwise each piece stores its partial block and the last piece to finish
// (per-index ticket) adds the partial blocks in piece order, so the result
// is deterministic.  Arithmetic:
//   GB_F32 : FP32 products of the hi parts, FP32 sums (per tile, then into
//            the running sum): the blocks of the mixed-precision operator;
//   GB_DF  : double-float products and sums (df.cuh) of hi + lo, or of the
//            FP64 copy split into hi + lo: FP64-accurate blocks, stored FP64.
//
// gram_apply_kernel: Yhat1(i,:) = C_i Xhat(i,:)', one warp per index, lanes
// over the output column j, reading row k of C_i (= column k, C_i is
// symmetric) coalesced for k = 0..r-1.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "df.cuh"
#include "launch.h"

namespace cphifi {
namespace {

enum { GB_F32 = 0, GB_DF = 1 };

template <int MODE>
struct GbTypes;
template <>
struct GbTypes<GB_F32> { using Acc = float; using Out = float; };
template <>
struct GbTypes<GB_DF> { using Acc = df; using Out = double; };

__device__ __forceinline__ void gb_fma(float& a, float x, float xl, float y, float yl) {
  (void)xl;
  (void)yl;
  a = fmaf(x, y, a);
}
__device__ __forceinline__ void gb_fma(df& a, float x, float xl, float y, float yl) {
  df_acc_prod(a, df{x, xl}, df{y, yl});
}
__device__ __forceinline__ void gb_zero(float& a) { a = 0.f; }
__device__ __forceinline__ void gb_zero(df& a) { a = df{0.f, 0.f}; }
__device__ __forceinline__ void gb_add(float& a, float b) { a += b; }
__device__ __forceinline__ void gb_add(df& a, df b) { df_acc_add(a, df_norm(b)); }
__device__ __forceinline__ float gb_out(float a) { return a; }
__device__ __forceinline__ double gb_out(df a) { return df_to_double(df_norm(a)); }

// pl: pieces of the Gram decomposition; npieces is read from np_dev (the
// piece-count scan's total) and clamped to pl.npieces.  zhi: the FP32 pair
// (tiles [hi | lo], stride 64 r) or NULL with z64 (FP64 copy, stride 32 r).
template <int MODE, int RP>
__global__ void __launch_bounds__(256) gram_build_kernel(PieceList pl, const int32_t* np_dev,
                                                         const float* __restrict__ zhi,
                                                         const double* __restrict__ z64, int r,
                                                         typename GbTypes<MODE>::Out* partial,
                                                         typename GbTypes<MODE>::Out* C,
                                                         const int* gate) {
  using Acc = typename GbTypes<MODE>::Acc;
  using Out = typename GbTypes<MODE>::Out;
  constexpr int T = RP / 16;
  constexpr int LD = RP + 4;  // staged row pitch (floats)
  __shared__ __align__(16) float zs[32 * LD];
  __shared__ __align__(16) float zl[MODE == GB_DF ? 32 * LD : 4];
  __shared__ int s_last;
  if (gate && *gate) return;
  const int npieces = min(pl.npieces, *np_dev);
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const bool upper = ty <= tx;
  const int64_t rr = (int64_t)r * r;
  for (int p = blockIdx.x; p < npieces; p += gridDim.x) {
    const int seg = pl.seg[p];
    const int b = pl.beg[p], e = pl.end[p];
    Acc acc[T][T];
#pragma unroll
    for (int a = 0; a < T; ++a)
#pragma unroll
      for (int c = 0; c < T; ++c) gb_zero(acc[a][c]);
    for (int t0 = b & ~31; t0 < e; t0 += 32) {
      __syncthreads();
      for (int idx = tid; idx < 32 * RP; idx += 256) {
        const int j = idx >> 5, l = idx & 31;
        const int64_t g = (int64_t)t0 + l;
        const bool in = j < r && g >= b && g < e;
        float h = 0.f, lo = 0.f;
        if (in) {
          if (zhi) {
            const int64_t base = zidx(g, j, 64 * (int64_t)r);
            h = __ldcs(zhi + base);
            if constexpr (MODE == GB_DF) lo = __ldcs(zhi + base + 32 * (int64_t)r);
          } else {
            const df v = df_from_double(__ldcs(z64 + zidx(g, j, 32 * (int64_t)r)));
            h = v.hi;
            lo = v.lo;
          }
        }
        zs[l * LD + j] = h;
        if constexpr (MODE == GB_DF) zl[l * LD + j] = lo;
      }
      __syncthreads();
      if (upper) {
        Acc part[T][T];
#pragma unroll
        for (int a = 0; a < T; ++a)
#pragma unroll
          for (int c = 0; c < T; ++c) gb_zero(part[a][c]);
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
          float x[T], y[T], xl[T], yl[T];
#pragma unroll
          for (int a = 0; a < T; ++a) {
            x[a] = zs[l * LD + ty * T + a];
            y[a] = zs[l * LD + tx * T + a];
            if constexpr (MODE == GB_DF) {
              xl[a] = zl[l * LD + ty * T + a];
              yl[a] = zl[l * LD + tx * T + a];
            } else {
              xl[a] = yl[a] = 0.f;
            }
          }
#pragma unroll
          for (int a = 0; a < T; ++a)
#pragma unroll
            for (int c = 0; c < T; ++c) gb_fma(part[a][c], x[a], xl[a], y[c], yl[c]);
        }
#pragma unroll
        for (int a = 0; a < T; ++a)
#pragma unroll
          for (int c = 0; c < T; ++c) gb_add(acc[a][c], part[a][c]);
      }
    }
    // write the upper tile (and its mirror image) of the piece's block
    const int np = pl.seg_count[seg];
    Out* dst = np == 1 ? C + (int64_t)seg * rr : partial + (int64_t)p * rr;
    if (upper) {
#pragma unroll
      for (int a = 0; a < T; ++a)
#pragma unroll
        for (int c = 0; c < T; ++c) {
          const int j = ty * T + a, k = tx * T + c;
          if (j < r && k < r && j <= k) {
            const Out v = gb_out(acc[a][c]);
            dst[(int64_t)j * r + k] = v;
            dst[(int64_t)k * r + j] = v;
          }
        }
    }
    if (np > 1) {
      __threadfence();
      __syncthreads();
      if (tid == 0) s_last = atomicAdd(&pl.seg_ticket[seg], 1u) == (unsigned)(np - 1);
      __syncthreads();
      if (s_last) {
        __threadfence();
        const int f = pl.seg_first[seg];
        for (int64_t t = tid; t < rr; t += 256) {
          Out sum = Out(0);
          for (int k = 0; k < np; ++k) sum += __ldcg(&partial[(int64_t)(f + k) * rr + t]);
          C[(int64_t)seg * rr + t] = sum;
        }
        if (tid == 0) pl.seg_ticket[seg] = 0u;
      }
    }
  }
}

// Yhat1(i, j) = sum_k C_i(k, j) Xhat(i, k) for every index i: warp per index.
template <typename TC, typename TX, typename TA>
__global__ void __launch_bounds__(256) gram_apply_kernel(const TC* __restrict__ C, int n, int r,
                                                         const TX* __restrict__ Xh, int64_t xld,
                                                         TX* __restrict__ Y, int64_t yld,
                                                         const DevScalars* skip) {
  if (dev_skip(skip)) return;
  const int lane = threadIdx.x & 31;
  const int64_t rr = (int64_t)r * r;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
       i += (gridDim.x * blockDim.x) >> 5) {
    const TC* Ci = C + (int64_t)i * rr;
    TA y0 = TA(0), y1 = TA(0);
    for (int k = 0; k < r; ++k) {
      const TA xk = (TA)Xh[(int64_t)k * xld + i];
      if (lane < r) y0 += (TA)Ci[(int64_t)k * r + lane] * xk;
      if (lane + 32 < r) y1 += (TA)Ci[(int64_t)k * r + lane + 32] * xk;
    }
    if (lane < r) Y[(int64_t)lane * yld + i] = (TX)y0;
    if (lane + 32 < r) Y[(int64_t)(lane + 32) * yld + i] = (TX)y1;
  }
}

// The FP32 blocks as a register-tiled segmented SYRK.  A block takes a piece;
// its 8 warps take the piece's 32-observation tiles in turn (warp w: tiles w,
// w + 8, ...), each staging its own tile in its own region of shared memory
// (observation-major rows, coalesced loads; only __syncwarp, so a warp
// waiting for its loads does not hold up the others).  Within a warp, lane
// u < U = G (G + 1) / 2 (G = RP / 8) owns the 8 x 8 tile (ti, tj), ti <= tj,
// of the upper triangle: per observation 2 + 2 128-bit shared loads feed 64
// multiply-adds.  At the end of the piece the 8 warps' partial blocks are
// added in warp order through shared memory.
template <int RP>
__global__ void __launch_bounds__(256, 2) gram_build_f32_tiled_kernel(PieceList pl,
                                                                      const int32_t* np_dev,
                                                                      const float* __restrict__ zhi,
                                                                      int r, float* partial,
                                                                      float* C) {
  // staged row pitch: 4 padding floats after every 32 columns, so that the
  // 8-float column groups a phase of 8 lanes loads fall in distinct banks
  constexpr int G = RP / 8, U = G * (G + 1) / 2, LD = RP + 4 * (RP / 32) + 8;
  static_assert(U <= 32, "one warp holds the upper triangle's 8 x 8 tiles");
  extern __shared__ __align__(16) float gsm[];  // 8 x 32 x LD staged values, then 8 x RP x RP
  __shared__ int s_last;
  const int npieces = min(pl.npieces, *np_dev);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // lane -> upper-triangle tile (ti, tj)
  int ti = 0, tj = 0;
  {
    int u = lane, row = 0;
    while (row < G && u >= G - row) { u -= G - row; ++row; }
    ti = row;
    tj = row + u;
  }
  const bool act = lane < U;
  const int xo = ti * 8 + 4 * (ti >> 2), yo = tj * 8 + 4 * (tj >> 2);
  const int64_t rr = (int64_t)r * r;
  const int64_t ts = 64 * (int64_t)r;  // tile stride of the FP32 pair
  float* zt = gsm + warp * 32 * LD;
  for (int p = blockIdx.x; p < npieces; p += gridDim.x) {
    const int seg = pl.seg[p];
    const int b = pl.beg[p], e = pl.end[p];
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
    for (int t0 = (b & ~31) + 32 * warp; t0 < e; t0 += 256) {
      // stage observations t0 .. t0 + 31 (lane = observation), zero outside
      // [b, e) and j >= r
      const int64_t g = (int64_t)t0 + lane;
      const bool in = g >= b && g < e;
      const float* src = zhi + (g >> 5) * ts + (g & 31);
      __syncwarp();
#pragma unroll 4
      for (int j = 0; j < RP; ++j) {
        const float v = (in && j < r) ? __ldcs(src + 32 * (int64_t)j) : 0.f;
        zt[lane * LD + j + 4 * (j >> 5)] = v;
      }
      __syncwarp();
      if (act) {
#pragma unroll 2
        for (int l = 0; l < 32; ++l) {
          const float4 x0 = *reinterpret_cast<const float4*>(zt + l * LD + xo);
          const float4 x1 = *reinterpret_cast<const float4*>(zt + l * LD + xo + 4);
          const float4 y0 = *reinterpret_cast<const float4*>(zt + l * LD + yo);
          const float4 y1 = *reinterpret_cast<const float4*>(zt + l * LD + yo + 4);
          const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
          const float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(xv[a], yv[c], acc[a][c]);
        }
      }
    }
    // the 8 warps' partial blocks, added in warp order
    __syncthreads();
    float* red = gsm;  // 8 x RP x RP
    if (act) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c)
          red[(warp * RP + ti * 8 + a) * RP + tj * 8 + c] = acc[a][c];
    }
    __syncthreads();
    const int np = pl.seg_count[seg];
    float* dst = np == 1 ? C + (int64_t)seg * rr : partial + (int64_t)p * rr;
    for (int t = tid; t < RP * RP; t += 256) {
      const int j = t / RP, k = t % RP;
      if (j < r && k < r && (j >> 3) <= (k >> 3)) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) v += red[(w * RP + j) * RP + k];
        // within a diagonal 8 x 8 tile both (j, k) and (k, j) were accumulated;
        // the upper one is written to both places
        if (j <= k) {
          dst[(int64_t)j * r + k] = v;
          dst[(int64_t)k * r + j] = v;
        }
      }
    }
    __syncthreads();  // red is read before the next piece stages over it
    if (np > 1) {
      __threadfence();
      __syncthreads();
      if (tid == 0) s_last = atomicAdd(&pl.seg_ticket[seg], 1u) == (unsigned)(np - 1);
      __syncthreads();
      if (s_last) {
        __threadfence();
        const int f = pl.seg_first[seg];
        for (int64_t t = tid; t < rr; t += 256) {
          float sum = 0.f;
          for (int k = 0; k < np; ++k) sum += __ldcg(&partial[(int64_t)(f + k) * rr + t]);
          C[(int64_t)seg * rr + t] = sum;
        }
        if (tid == 0) pl.seg_ticket[seg] = 0u;
      }
    }
  }
}

template <int RP>
cudaError_t build_f32_tiled(const PieceList& pl, const int32_t* np_dev, int grid,
                            const float* zhi, int r, float* partial, float* C, cudaStream_t st) {
  const size_t smem = (size_t)std::max(8 * 32 * (RP + 4 * (RP / 32) + 8), 8 * RP * RP) *
                      sizeof(float);
  const cudaError_t e = cudaFuncSetAttribute(gram_build_f32_tiled_kernel<RP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
  if (e != cudaSuccess) return e;
  gram_build_f32_tiled_kernel<RP><<<grid, 256, smem, st>>>(pl, np_dev, zhi, r, partial, C);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t build_by_rank(const PieceList& pl, const int32_t* np_dev, int grid, const float* zhi,
                          const double* z64, int r, typename GbTypes<MODE>::Out* partial,
                          typename GbTypes<MODE>::Out* C, const int* gate, cudaStream_t st) {
  if (r <= 16)
    gram_build_kernel<MODE, 16><<<grid, 256, 0, st>>>(pl, np_dev, zhi, z64, r, partial, C, gate);
  else if (r <= 32)
    gram_build_kernel<MODE, 32><<<grid, 256, 0, st>>>(pl, np_dev, zhi, z64, r, partial, C, gate);
  else if (r <= 48)
    gram_build_kernel<MODE, 48><<<grid, 256, 0, st>>>(pl, np_dev, zhi, z64, r, partial, C, gate);
  else if (r <= 64)
    gram_build_kernel<MODE, 64><<<grid, 256, 0, st>>>(pl, np_dev, zhi, z64, r, partial, C, gate);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gram_build_f32(const PieceList& pl, const int32_t* np_dev, int grid,
                                  const float* zhi, int r, float* partial, float* C,
                                  cudaStream_t st) {
  if (pl.npieces == 0) return cudaSuccess;
  if (r <= 16) return build_f32_tiled<16>(pl, np_dev, grid, zhi, r, partial, C, st);
  if (r <= 32) return build_f32_tiled<32>(pl, np_dev, grid, zhi, r, partial, C, st);
  if (r <= 48) return build_f32_tiled<48>(pl, np_dev, grid, zhi, r, partial, C, st);
  return build_by_rank<GB_F32>(pl, np_dev, grid, zhi, nullptr, r, partial, C, nullptr, st);
}

cudaError_t launch_gram_build_df(const PieceList& pl, const int32_t* np_dev, int grid,
                                 const float* zhi, const double* z64, int r, double* partial,
                                 double* C, cudaStream_t st) {
  if (pl.npieces == 0) return cudaSuccess;
  return build_by_rank<GB_DF>(pl, np_dev, grid, zhi, z64, r, partial, C, nullptr, st);
}

cudaError_t launch_gram_apply_f32(const float* C, int n, int r, const float* Xh, int64_t xld,
                                  float* Y, int64_t yld, const DevScalars* skip,
                                  cudaStream_t st) {
  const int blocks = (n + 7) / 8;
  gram_apply_kernel<float, float, float><<<blocks, 256, 0, st>>>(C, n, r, Xh, xld, Y, yld, skip);
  return cudaGetLastError();
}

cudaError_t launch_gram_apply_f64(const double* C, int n, int r, const double* Xh, int64_t xld,
                                  double* Y, int64_t yld, const DevScalars* skip,
                                  cudaStream_t st) {
  const int blocks = (n + 7) / 8;
  gram_apply_kernel<double, double, double><<<blocks, 256, 0, st>>>(C, n, r, Xh, xld, Y, yld,
                                                                    skip);
  return cudaGetLastError();
}

}  // namespace cphifi
