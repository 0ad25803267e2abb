// Kernels of the alternating fit around the kernel-mode solve (§2): the
// observation lists kept in sorted order, the per-mode sort for the
// finite-mode updates, the CP-ALS row update (r x r normal equations and
// Cholesky per row, FP64), and the fit error of the model.
#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.h"

namespace cphifi {

// ---------------------------------------------- sorted observation lists --
// kidx_s[l] = keys[l] (the sorted kernel indices), and the other-mode indices
// and values of observation perm[l] (or l when perm is NULL).
__global__ void keep_obs_kernel(int64_t q, int d_other, const uint32_t* __restrict__ keys,
                                const int32_t* __restrict__ perm, const int32_t* __restrict__ oidx,
                                const double* __restrict__ vals, int32_t* __restrict__ kidx_s,
                                int32_t* __restrict__ oidx_s, double* __restrict__ vals_s,
                                const int* gate) {
  if (gate && *gate) return;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < q;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = perm ? (int64_t)perm[l] : l;
    kidx_s[l] = (int32_t)keys[l];
    vals_s[l] = vals[src];
    for (int m = 0; m < d_other; ++m) oidx_s[l * d_other + m] = oidx[src * d_other + m];
  }
}

cudaError_t launch_keep_obs(int64_t q, int d_other, const uint32_t* keys, const int32_t* perm,
                            const int32_t* oidx, const double* vals, int32_t* kidx_s,
                            int32_t* oidx_s, double* vals_s, const int* gate, cudaStream_t st) {
  if (q == 0) return cudaSuccess;
  int64_t b = (q + 255) / 256;
  if (b > 8192) b = 8192;
  keep_obs_kernel<<<(int)b, 256, 0, st>>>(q, d_other, keys, perm, oidx, vals, kidx_s, oidx_s,
                                          vals_s, gate);
  return cudaGetLastError();
}

// keys[l] = oidx_s[l * d_other + m]: the sort keys of finite mode m.
__global__ void mode_keys_kernel(int64_t q, int d_other, int m, const int32_t* __restrict__ oidx_s,
                                 uint32_t* __restrict__ keys) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < q;
       l += (int64_t)gridDim.x * blockDim.x)
    keys[l] = (uint32_t)oidx_s[l * d_other + m];
}

cudaError_t launch_mode_keys(int64_t q, int d_other, int m, const int32_t* oidx_s, uint32_t* keys,
                             cudaStream_t st) {
  if (q == 0) return cudaSuccess;
  int64_t b = (q + 255) / 256;
  if (b > 8192) b = 8192;
  mode_keys_kernel<<<(int)b, 256, 0, st>>>(q, d_other, m, oidx_s, keys);
  return cudaGetLastError();
}

// ------------------------------------------------- CP-ALS row update ------
// Block per row i of finite mode m (grid-stride over rows).  The row's
// observations (in the mode-m order, perm_m) are taken 32 at a time: their
// vectors z_l = A_k(i_l,:) o prod_{m' != m} A_m'(i_m'^l,:) are formed in
// shared memory, and thread t accumulates the pairs (j, k), j <= k, numbered
// t, t + blockDim, ... of G_i = sum z z' and, for t < r, h_i(t) = sum t_l z_l(t).
// G_i then goes to shared memory, gets the ridge 1e-12 trace(G_i) when the
// row has fewer than r observations, and is factored by a right-looking
// Cholesky; two triangular solves give the new row.  Rows without
// observations, with a zero trace, or not positive definite keep their old
// values.  All sums are FP64 in a fixed order.
constexpr int kAlsChunk = 32;
constexpr int kAlsThreads = 256;

template <int RP>
__global__ void __launch_bounds__(kAlsThreads)
als_row_kernel(int n_m, int m, int d_other, int r, int n, const int64_t* __restrict__ row_ptr_m,
               const int32_t* __restrict__ perm_m, const int32_t* __restrict__ kidx_s,
               const int32_t* __restrict__ oidx_s, const double* __restrict__ vals_s,
               const double* __restrict__ Ak, const double* const* __restrict__ factors,
               const int64_t* __restrict__ sizes, double* __restrict__ Anew,
               int* __restrict__ nfail) {
  constexpr int NP = (RP * (RP + 1) / 2 + kAlsThreads - 1) / kAlsThreads;
  // the chunk vectors and, after the sums, the matrix share one buffer
  constexpr int ZS = kAlsChunk * RP, GS = RP * (RP + 1);
  __shared__ double buf[ZS > GS ? ZS : GS];
  __shared__ double ts[kAlsChunk];
  __shared__ double hv[RP];
  double (*zs)[RP] = reinterpret_cast<double (*)[RP]>(buf);
  double (*G)[RP + 1] = reinterpret_cast<double (*)[RP + 1]>(buf);
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int npairs = r * (r + 1) / 2;
  // pair index -> (j, k), j <= k, row-wise over the upper triangle
  int pj[NP], pk[NP];
#pragma unroll
  for (int u = 0; u < NP; ++u) {
    int p = tid + u * kAlsThreads, j = 0;
    if (p >= npairs) { pj[u] = -1; pk[u] = -1; continue; }
    while (p >= r - j) { p -= r - j; ++j; }
    pj[u] = j;
    pk[u] = j + p;
  }
  for (int i = blockIdx.x; i < n_m; i += gridDim.x) {
    const int64_t beg = row_ptr_m[i], end = row_ptr_m[i + 1];
    double acc[NP];
#pragma unroll
    for (int u = 0; u < NP; ++u) acc[u] = 0.0;
    double hacc = 0.0;
    for (int64_t c0 = beg; c0 < end; c0 += kAlsChunk) {
      const int cnt = (int)min((int64_t)kAlsChunk, end - c0);
      __syncthreads();
      for (int e = tid; e < kAlsChunk * r; e += kAlsThreads) {
        const int o = e / r, j = e - (e / r) * r;
        double z = 0.0;
        if (o < cnt) {
          const int64_t s = perm_m[c0 + o];
          z = Ak[kidx_s[s] + (int64_t)n * j];
          for (int m2 = 0; m2 < d_other; ++m2)
            if (m2 != m) z *= factors[m2][oidx_s[s * d_other + m2] + sizes[m2] * j];
          if (j == 0) ts[o] = vals_s[s];
        } else if (j == 0) {
          ts[o] = 0.0;
        }
        zs[o][j] = z;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < NP; ++u) {
        if (pj[u] < 0) continue;
        double a = acc[u];
        for (int o = 0; o < kAlsChunk; ++o) a = fma(zs[o][pj[u]], zs[o][pk[u]], a);
        acc[u] = a;
      }
      if (tid < r)
        for (int o = 0; o < kAlsChunk; ++o) hacc = fma(ts[o], zs[o][tid], hacc);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NP; ++u)
      if (pj[u] >= 0) {
        G[pj[u]][pk[u]] = acc[u];
        G[pk[u]][pj[u]] = acc[u];
      }
    if (tid < r) hv[tid] = hacc;
    if (tid == 0) bad = 0;
    __syncthreads();
    const int64_t count = end - beg;
    double tr = 0.0;
    for (int j = 0; j < r; ++j) tr += G[j][j];  // every thread, same order
    bool keep = count == 0 || !(tr > 0.0);
    if (!keep && count < r) {
      __syncthreads();
      if (tid < r) G[tid][tid] += 1e-12 * tr;
      __syncthreads();
    }
    // right-looking Cholesky, lower triangle in place
    for (int c = 0; c < r && !keep; ++c) {
      if (tid == 0) {
        const double piv = G[c][c];
        if (!(piv > 0.0) || !isfinite(piv)) bad = 1;
        else G[c][c] = sqrt(piv);
      }
      __syncthreads();
      if (bad) { keep = true; break; }
      const double lcc = G[c][c];
      for (int i2 = c + 1 + tid; i2 < r; i2 += kAlsThreads) G[i2][c] /= lcc;
      __syncthreads();
      const int rem = r - c - 1;
      for (int e = tid; e < rem * rem; e += kAlsThreads) {
        const int i2 = c + 1 + e / rem, j2 = c + 1 + e % rem;
        if (j2 <= i2) G[i2][j2] -= G[i2][c] * G[j2][c];
      }
      __syncthreads();
    }
    if (keep) {
      if (tid < r) Anew[i + (int64_t)n_m * tid] = factors[m][i + sizes[m] * tid];
      if (tid == 0 && count > 0) atomicAdd(nfail, 1);
    } else if (tid == 0) {
      // L y = h, L' a = y (sequential: r <= 64)
      for (int j = 0; j < r; ++j) {
        double v = hv[j];
        for (int p = 0; p < j; ++p) v -= G[j][p] * hv[p];
        hv[j] = v / G[j][j];
      }
      for (int j = r - 1; j >= 0; --j) {
        double v = hv[j];
        for (int p = j + 1; p < r; ++p) v -= G[p][j] * hv[p];
        hv[j] = v / G[j][j];
      }
    }
    __syncthreads();
    if (!keep && tid < r) Anew[i + (int64_t)n_m * tid] = hv[tid];
    __syncthreads();
  }
}

cudaError_t launch_als_rows(int n_m, int m, int d_other, int r, int n, const int64_t* row_ptr_m,
                            const int32_t* perm_m, const int32_t* kidx_s, const int32_t* oidx_s,
                            const double* vals_s, const double* Ak, const double* const* factors,
                            const int64_t* sizes, double* Anew, int* nfail, int num_sms,
                            cudaStream_t st) {
  if (n_m == 0) return cudaSuccess;
  int blocks = n_m < num_sms * 4 ? n_m : num_sms * 4;
#define CPHIFI_ALS(RPV)                                                                        \
  als_row_kernel<RPV><<<blocks, kAlsThreads, 0, st>>>(n_m, m, d_other, r, n, row_ptr_m, perm_m, \
                                                      kidx_s, oidx_s, vals_s, Ak, factors,     \
                                                      sizes, Anew, nfail)
  if (r <= 8) CPHIFI_ALS(8);
  else if (r <= 16) CPHIFI_ALS(16);
  else if (r <= 32) CPHIFI_ALS(32);
  else if (r <= 48) CPHIFI_ALS(48);
  else if (r <= 64) CPHIFI_ALS(64);
  else return cudaErrorInvalidValue;
#undef CPHIFI_ALS
  return cudaGetLastError();
}

// --------------------------------------------------------- fit error ------
// out[0] = sum_l (t_l - m_l)^2, out[1] = sum_l t_l^2 with
// m_l = sum_j A_k(i_l, j) prod_m A_m(i_m^l, j) (FP64, deterministic sums).
__global__ void __launch_bounds__(256)
fit_kernel(int64_t q, int d_other, int r, int n, const int32_t* __restrict__ kidx_s,
           const int32_t* __restrict__ oidx_s, const double* __restrict__ vals_s,
           const double* __restrict__ Ak, const double* const* __restrict__ factors,
           const int64_t* __restrict__ sizes, RedScratch red, double* out) {
  double v[2] = {0.0, 0.0};
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < q;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = kidx_s[l];
    double mdl = 0.0;
    for (int j = 0; j < r; ++j) {
      double z = Ak[i + (int64_t)n * j];
      for (int m = 0; m < d_other; ++m) z *= factors[m][oidx_s[l * d_other + m] + sizes[m] * j];
      mdl += z;
    }
    const double t = vals_s[l];
    v[0] = fma(t - mdl, t - mdl, v[0]);
    v[1] = fma(t, t, v[1]);
  }
  double tot[2];
  if (grid_sum_last<2>(v, red, tot)) {
    out[0] = tot[0];
    out[1] = tot[1];
  }
}

cudaError_t launch_fit(int64_t q, int d_other, int r, int n, const int32_t* kidx_s,
                       const int32_t* oidx_s, const double* vals_s, const double* Ak,
                       const double* const* factors, const int64_t* sizes, RedScratch red,
                       double* out, int num_sms, cudaStream_t st) {
  int64_t b = (q + 255) / 256;
  if (b > (int64_t)num_sms * 4) b = (int64_t)num_sms * 4;
  if (b > kRedMaxBlocks) b = kRedMaxBlocks;
  if (b < 1) b = 1;
  fit_kernel<<<(int)b, 256, 0, st>>>(q, d_other, r, n, kidx_s, oidx_s, vals_s, Ak, factors, sizes,
                                     red, out);
  return cudaGetLastError();
}

}  // namespace cphifi
