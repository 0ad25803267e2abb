// Kernel matrices from design points (§2: the kernel mode's factor lives in
// an RKHS with kernel k, K(i, j) = k(x_i, x_j) on the mode's points).
//
// kpoints_build_kernel writes K itself (FP64, both triangles) for the
// one-time eigendecomposition of Eq. eigK.  kpoints_apply_kernel computes
// Y = K X for an n x r X without K in memory: each block owns 64 rows of Y
// and a range of columns of K, which it walks in tiles of 32, generating each
// 64 x 32 tile of K from the points in shared memory (one exp per entry) and
// multiplying it with the matching 32 x r tile of X.  The product then reads
// only the points and X (n (dim + r) values) instead of n^2 entries: it is
// bound by the arithmetic (n^2 r multiply-adds and n^2 exponentials), not by
// HBM.  With n / 64 row blocks alone a grid would cover few SMs (32 blocks at
// n = 2048: a fifth of the GPU), so the column range is split over
// blockIdx.y as well; the splits' partial products are then added in split
// order (kpoints_combine_kernel), so the result does not depend on the
// timing of the blocks.
//
// Kernels: Gaussian k(x, y) = exp(-|x - y|^2 / (2 s^2)) and Matern-3/2
// k(x, y) = (1 + sqrt(3) d / s) exp(-sqrt(3) d / s), d = |x - y|, with s the
// bandwidth (length scale); points are rows of an n x dim row-major array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cphifi.h"
#include "launch.h"

namespace cphifi {
namespace {

template <typename T>
__device__ __forceinline__ T kp_exp(T v);
template <>
__device__ __forceinline__ double kp_exp<double>(double v) { return exp(v); }
template <>
__device__ __forceinline__ float kp_exp<float>(float v) { return __expf(v); }

template <typename T>
__device__ __forceinline__ T kp_eval(int kind, T d2, T inv_bw) {
  if (kind == CPHIFI_KERNEL_GAUSSIAN) return kp_exp<T>(T(-0.5) * d2 * inv_bw * inv_bw);
  const T u = T(1.7320508075688772) * sqrt(d2) * inv_bw;  // sqrt(3) d / s
  return (T(1) + u) * kp_exp<T>(-u);
}

template <typename T>
__device__ __forceinline__ T kp_dist2(const double* __restrict__ pts, int dim, int i, int j) {
  T d2 = T(0);
  for (int c = 0; c < dim; ++c) {
    const T t = (T)(pts[(int64_t)i * dim + c] - pts[(int64_t)j * dim + c]);
    d2 += t * t;
  }
  return d2;
}

__global__ void kpoints_build_kernel(const double* __restrict__ pts, int n, int dim, int kind,
                                     double inv_bw, double* __restrict__ K) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    K[e] = kp_eval<double>(kind, kp_dist2<double>(pts, dim, i, j), inv_bw);
  }
}

// Y(i, c) = sum_k K(i, k) X(k, c), X and Y column-major (ld n), T the
// arithmetic (FP64, or FP32 with the hardware exponential).  Block: 256
// threads = 64 rows x 4 column groups; thread (row, g) accumulates columns
// g, g + 4, ... (RP / 4 of them).
template <typename T, int RP>
__global__ void __launch_bounds__(256) kpoints_apply_kernel(const double* __restrict__ pts, int n,
                                                            int dim, int kind, double inv_bw,
                                                            int r, const double* __restrict__ X,
                                                            double* __restrict__ Y, int kchunk) {
  constexpr int TM = 64, TK = 32, CG = 4, CPT = RP / CG;
  __shared__ T kt[TK][TM + 1];  // K tile, column-major within the tile
  __shared__ T xt[TK][RP];
  const int row = threadIdx.x % TM, g = threadIdx.x / TM;
  const int i0 = blockIdx.x * TM;
  const int i = i0 + row;
  T acc[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) acc[c] = T(0);
  const T ib = (T)inv_bw;
  const int kbeg = blockIdx.y * kchunk, kend = min(n, kbeg + kchunk);
  Y += (int64_t)blockIdx.y * n * r;  // this split's partial product
  for (int k0 = kbeg; k0 < kend; k0 += TK) {
    __syncthreads();
    for (int e = threadIdx.x; e < TM * TK; e += blockDim.x) {
      const int a = e % TM, b = e / TM;  // row i0 + a, column k0 + b
      const int ii = i0 + a, kk = k0 + b;
      kt[b][a] = (ii < n && kk < kend) ? kp_eval<T>(kind, kp_dist2<T>(pts, dim, ii, kk), ib) : T(0);
    }
    for (int e = threadIdx.x; e < TK * RP; e += blockDim.x) {
      const int b = e % TK, c = e / TK;
      const int kk = k0 + b;
      xt[b][c] = (kk < kend && c < r) ? (T)X[(int64_t)c * n + kk] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int b = 0; b < TK; ++b) {
      const T kv = kt[b][row];
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[c] += kv * xt[b][g + CG * c];
    }
  }
  if (i < n) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int col = g + CG * c;
      if (col < r) Y[(int64_t)col * n + i] = (double)acc[c];
    }
  }
}

// Y(t) = sum over the splits, in order, of part[s n r + t].
__global__ void kpoints_combine_kernel(const double* __restrict__ part, int nsplit, int64_t nr,
                                       double* __restrict__ Y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nr;
       t += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int s = 0; s < nsplit; ++s) a += part[s * nr + t];
    Y[t] = a;
  }
}

template <typename T>
cudaError_t apply_by_rank(const double* pts, int n, int dim, int kind, double inv_bw, int r,
                          const double* X, double* Y, int nsplit, cudaStream_t st) {
  int kchunk = (n + nsplit - 1) / nsplit;
  kchunk = (kchunk + 31) / 32 * 32;
  const dim3 grid((n + 63) / 64, (n + kchunk - 1) / kchunk);
  if (r <= 8)
    kpoints_apply_kernel<T, 8><<<grid, 256, 0, st>>>(pts, n, dim, kind, inv_bw, r, X, Y, kchunk);
  else if (r <= 16)
    kpoints_apply_kernel<T, 16><<<grid, 256, 0, st>>>(pts, n, dim, kind, inv_bw, r, X, Y, kchunk);
  else if (r <= 32)
    kpoints_apply_kernel<T, 32><<<grid, 256, 0, st>>>(pts, n, dim, kind, inv_bw, r, X, Y, kchunk);
  else if (r <= 64)
    kpoints_apply_kernel<T, 64><<<grid, 256, 0, st>>>(pts, n, dim, kind, inv_bw, r, X, Y, kchunk);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_kpoints_build(const double* pts, int n, int dim, int kind, double bandwidth,
                                 double* K, cudaStream_t st) {
  const int64_t nn = (int64_t)n * n;
  const int blocks = (int)((nn + 255) / 256 < 4096 ? (nn + 255) / 256 : 4096);
  kpoints_build_kernel<<<blocks, 256, 0, st>>>(pts, n, dim, kind, 1.0 / bandwidth, K);
  return cudaGetLastError();
}

int kpoints_pick_split(int n, int num_sms) {
  // about two blocks per SM (the FP64 tile runs 4 per SM, the FP32 one 5),
  // each split at least 128 columns of K
  const int rows = (n + 63) / 64;
  int s = (2 * num_sms + rows - 1) / rows;
  s = std::min(s, std::max(1, n / 128));
  return std::max(1, std::min(s, 32));
}

cudaError_t launch_kpoints_apply(bool fp64, const double* pts, int n, int dim, int kind,
                                 double bandwidth, int r, const double* X, double* Y,
                                 int nsplit, double* part, cudaStream_t st) {
  if (n == 0 || r == 0) return cudaSuccess;
  if (nsplit < 1 || (nsplit > 1 && !part)) return cudaErrorInvalidValue;
  double* out = nsplit > 1 ? part : Y;
  cudaError_t e = fp64 ? apply_by_rank<double>(pts, n, dim, kind, 1.0 / bandwidth, r, X, out,
                                               nsplit, st)
                       : apply_by_rank<float>(pts, n, dim, kind, 1.0 / bandwidth, r, X, out,
                                              nsplit, st);
  if (e != cudaSuccess || nsplit == 1) return e;
  int kchunk = (n + nsplit - 1) / nsplit;
  kchunk = (kchunk + 31) / 32 * 32;
  const int used = (n + kchunk - 1) / kchunk;  // splits the grid actually had
  const int64_t nr = (int64_t)n * r;
  const int blocks = (int)std::min<int64_t>((nr + 255) / 256, 2048);
  kpoints_combine_kernel<<<blocks, 256, 0, st>>>(part, used, nr, Y);
  return cudaGetLastError();
}

}  // namespace cphifi
