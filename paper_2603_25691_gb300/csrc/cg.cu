// Small dense pieces of the solve: the Gram matrix V = Z'Z (§3), its
// eigendecomposition (Eq. eigV) by parallel cyclic Jacobi, the preconditioner
// diagonal D (§4.4.2), and the fused PCG vector kernels (the epilogue of the
// operator, the residual/solution updates with the preconditioner apply of
// Eq. fx, the direction update) with their deterministic grid reductions.
//
// The PCG runs in the eigenbasis of K (X = U_K Xbar).  There the operator of
// Eq. unaligned-infinite-1 reads
//   Abar xbar = D_K U_K' Yhat1(U_K D_K Xbar) + (lambda D_K + rho) .* Xbar
// and the preconditioner of Eq. fx reduces to the r x r part
//   Mbar^{-1} Xbar = ((Xbar U_V) .* D) U_V'.
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"

namespace cphifi {

// -------------------------------------------------------------- Gram V ----
// V(a, b) = prod_m sum_i A_m(i, a) A_m(i, b): one block per (a, b).
__global__ void gram_kernel(const double* const* __restrict__ factors,
                            const int64_t* __restrict__ sizes, int d_other, int r, double* V) {
  __shared__ double sm[32];
  const int a = blockIdx.x % r, b = blockIdx.x / r;
  double prod = 1.0;
  for (int m = 0; m < d_other; ++m) {
    const double* F = factors[m];
    const int64_t nm = sizes[m];
    double v[1] = {0.0};
    for (int64_t i = threadIdx.x; i < nm; i += blockDim.x) v[0] += F[a * nm + i] * F[b * nm + i];
    block_sum<1>(v, sm);
    __syncthreads();
    if (threadIdx.x == 0) sm[31] = v[0];
    __syncthreads();
    prod *= sm[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) V[a + (int64_t)r * b] = prod;
}

cudaError_t launch_gram(const double* const* factors_dev, const int64_t* sizes_dev, int d_other,
                        int r, double* V, cudaStream_t st) {
  gram_kernel<<<r * r, 256, 0, st>>>(factors_dev, sizes_dev, d_other, r, V);
  return cudaGetLastError();
}

// ------------------------------------------------------ Jacobi eig(V) -----
// One block.  Brent-Luk parallel ordering: each round rotates R/2 disjoint
// (p, q) pairs chosen by the round-robin (circle) schedule; R = r rounded up
// to even, the extra index being an isolated zero.  Rotation of
// Golub & Van Loan, Matrix Computations, §8.5 (symmetric Schur 2 x 2):
// tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1/sqrt(1 + t^2), s = t c, then A <- J'AJ and Q <- QJ.
//
// GB300 runs FP64 multiply-adds at 1/63 of the FP32 rate, and a sweep is
// ~6 R^2 (R - 1) multiply-adds on one SM, so the sweeps first run in FP32
// (to an off-diagonal Frobenius norm of ~1e-6 ||A||) and give a basis Q0;
// then B = Q0' V Q0 is formed in FP64 -- diagonal up to the FP32 error -- and
// FP64 sweeps on B, accumulating into Q = Q0 J, finish to an off-diagonal
// norm below 1e-14 ||V||_F (quadratic convergence: one or two sweeps).
// info = 1 if that target was not met within max_sweeps FP64 sweeps.
// Eigenvalues are left unsorted.
template <typename T>
__device__ void jacobi_sweeps(T* A, T* Q, T* cs, int* pq, int R, int max_sweeps, double tol2,
                              double* red, double* stats /* off, nrm */) {
  for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
    double v[2] = {0.0, 0.0};
    for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
      const int i = t % R, j = t / R;
      const double a = (double)A[t];
      v[1] += a * a;
      if (i != j) v[0] += a * a;
    }
    block_sum<2>(v, red);
    if (threadIdx.x == 0) { stats[0] = v[0]; stats[1] = v[1]; }
    __syncthreads();
    if (stats[0] <= tol2 * stats[1] || stats[0] == 0.0 || sweep == max_sweeps) break;
    for (int round = 0; round < R - 1; ++round) {
      for (int k = threadIdx.x; k < R / 2; k += blockDim.x) {
        int a, b;
        if (k == 0) { a = R - 1; b = round; }
        else { a = (round + k) % (R - 1); b = (round - k + R - 1) % (R - 1); }
        const int p = min(a, b), q = max(a, b);
        const T apq = A[p + R * q];
        T c = T(1), sn = T(0);
        if (apq != T(0)) {
          const T tau = (A[q + R * q] - A[p + R * p]) / (T(2) * apq);
          const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          c = T(1) / sqrt(T(1) + t * t);
          sn = t * c;
        }
        cs[2 * k] = c; cs[2 * k + 1] = sn;
        pq[2 * k] = p; pq[2 * k + 1] = q;
      }
      __syncthreads();
      // rows: (J'A)(p,:) = c A(p,:) - s A(q,:); (J'A)(q,:) = s A(p,:) + c A(q,:)
      for (int t = threadIdx.x; t < (R / 2) * R; t += blockDim.x) {
        const int k = t / R, col = t % R;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const T c = cs[2 * k], sn = cs[2 * k + 1];
        const T ap = A[p + R * col], aq = A[q + R * col];
        A[p + R * col] = c * ap - sn * aq;
        A[q + R * col] = sn * ap + c * aq;
      }
      __syncthreads();
      // columns of A and Q: (AJ)(:,p) = c A(:,p) - s A(:,q); (AJ)(:,q) = s A(:,p) + c A(:,q)
      for (int t = threadIdx.x; t < (R / 2) * R; t += blockDim.x) {
        const int k = t / R, row = t % R;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const T c = cs[2 * k], sn = cs[2 * k + 1];
        const T ap = A[row + R * p], aq = A[row + R * q];
        A[row + R * p] = c * ap - sn * aq;
        A[row + R * q] = sn * ap + c * aq;
        const T qp = Q[row + R * p], qq = Q[row + R * q];
        Q[row + R * p] = c * qp - sn * qq;
        Q[row + R * q] = sn * qp + c * qq;
      }
      __syncthreads();
    }
  }
}

__global__ void jacobi_kernel(const double* __restrict__ Vin, int r, double* dV, double* UV,
                              int max_sweeps, int* info) {
  extern __shared__ double smj[];
  const int R = r + (r & 1);
  double* A = smj;              // R x R, A[i + R j]
  double* Q = A + R * R;        // R x R
  double* Tm = Q + R * R;       // R x R (FP64 work)
  double* cs = Tm + R * R;      // R/2 x 2
  float* A32 = reinterpret_cast<float*>(cs + R);  // R x R
  float* Q32 = A32 + R * R;                       // R x R
  float* cs32 = Q32 + R * R;                      // R/2 x 2
  int* pq = reinterpret_cast<int*>(cs32 + R);     // R/2 x 2
  __shared__ double red[64];  // block_sum<2> scratch: 2 x 32
  __shared__ double stats[2];
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    const int i = t % R, j = t / R;
    const double v = (i < r && j < r) ? Vin[i + (int64_t)r * j] : 0.0;
    A[t] = v;
    A32[t] = (float)v;
    Q32[t] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  // FP32 sweeps: an approximate eigenbasis Q0
  jacobi_sweeps<float>(A32, Q32, cs32, pq, R, 40, 1e-12, red, stats);
  // Q0 is orthogonal only to FP32 accuracy: two Newton-Schulz steps
  // Q <- Q (3 I - Q'Q) / 2 in FP64 take ||I - Q'Q|| from ~1e-7 to rounding.
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) Q[t] = (double)Q32[t];
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    for (int t = threadIdx.x; t < R * R; t += blockDim.x) {  // Tm = (3 I - Q'Q) / 2
      const int i = t % R, j = t / R;
      double acc = 0.0;
      for (int k = 0; k < R; ++k) acc = fma(Q[k + R * i], Q[k + R * j], acc);
      Tm[t] = (i == j ? 1.5 : 0.0) - 0.5 * acc;
    }
    __syncthreads();
    // Q <- Q Tm: every thread first computes its entries (at most
    // R*R / blockDim = 16 for R <= 64 and 256 threads), then all write.
    double qn[16];
    int cnt = 0;
    for (int t = threadIdx.x; t < R * R; t += blockDim.x, ++cnt) {
      const int i = t % R, j = t / R;
      double acc = 0.0;
      for (int k = 0; k < R; ++k) acc = fma(Q[i + R * k], Tm[k + R * j], acc);
      qn[cnt] = acc;
    }
    __syncthreads();
    cnt = 0;
    for (int t = threadIdx.x; t < R * R; t += blockDim.x, ++cnt) Q[t] = qn[cnt];
    __syncthreads();
  }
  // B = Q' V Q in FP64 (V is still in A): Tm = V Q, then A = Q' Tm
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    const int i = t % R, j = t / R;
    double acc = 0.0;
    for (int k = 0; k < R; ++k) acc = fma(A[i + R * k], Q[k + R * j], acc);
    Tm[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) {
    const int i = t % R, j = t / R;
    double acc = 0.0;
    for (int k = 0; k < R; ++k) acc = fma(Q[k + R * i], Tm[k + R * j], acc);
    A[t] = acc;
  }
  __syncthreads();
  // FP64 sweeps on B, rotations accumulated into Q = Q0 J
  jacobi_sweeps<double>(A, Q, cs, pq, R, max_sweeps, 1e-28, red, stats);
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    const int i = t % r, j = t / r;
    UV[t] = Q[i + R * j];
  }
  for (int t = threadIdx.x; t < r; t += blockDim.x) dV[t] = A[t + R * t];
  if (threadIdx.x == 0)
    *info = (stats[0] <= 1e-28 * stats[1] || stats[0] == 0.0) ? 0 : 1;
}

cudaError_t launch_jacobi_eig(const double* V, int r, double* dV, double* UV, int max_sweeps,
                              int* info, cudaStream_t st) {
  const int R = r + (r & 1);
  const size_t smem = (size_t)(3 * R * R + R) * sizeof(double) +
                      (size_t)(2 * R * R + R) * sizeof(float) + (size_t)R * sizeof(int);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  jacobi_kernel<<<1, 256, smem, st>>>(V, r, dV, UV, max_sweeps, info);
  return cudaGetLastError();
}

// ------------------------------------------------------- D (Eq. fx) -------
// D(i, j) = 1 / (gamma D_V(j) D_K(i)^2 + lambda D_K(i) + rho), with round-off
// negative eigenvalues of the PSD K and V clamped to 0 here only.
__global__ void build_D_kernel(const double* __restrict__ dK, const double* __restrict__ dV,
                               int n, int r, double gamma, double lam, double rho, double* D64,
                               float* D32) {
  const int64_t total = (int64_t)n * r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    const double k = fmax(dK[i], 0.0), v = fmax(dV[j], 0.0);
    const double d = 1.0 / (gamma * v * k * k + lam * k + rho);
    D64[t] = d;
    if (D32) D32[t] = (float)d;
  }
}

cudaError_t launch_build_D(const double* dK, const double* dV, int n, int r, double gamma,
                           double lam, double rho, double* D64, float* D32, cudaStream_t st) {
  const int64_t total = (int64_t)n * r;
  const int blocks = (int)((total + 255) / 256 < 2048 ? (total + 255) / 256 : 2048);
  build_D_kernel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(dK, dV, n, r, gamma, lam, rho, D64, D32);
  return cudaGetLastError();
}

// ------------------------------------------------- operator epilogue ------
// Sums the split partial products and applies the elementwise tail.  CM_APPLY
// also forms (p, Ap) and, in its last block, alpha = rz / pAp; CM_RESID and
// CM_TRUE form ||b - A x||^2 and, in their last block, decide convergence on
// the FP64 true residual (CM_RESID also makes it the recurrence residual).
//
// The partials are dead once summed, and each element is read by one thread
// only: every warp drops from L2, without write-back, the 128-byte lines of
// partials that lie wholly inside what it has read (discard.global.L2).  Left
// dirty, those lines (tens to hundreds of MB) are written back while the next
// observation pass streams Zhat, and slow it: a 400 MB dirty buffer in L2
// made a double-float pass at n = 8000, q = 5e7 take 5.5 ms instead of 3.3.

// Drops the lines of the split partials C[k stride + b0, k stride + e0)
// (k < ns) that lie wholly inside that range; called by the whole warp after
// it has read those elements.
template <typename TC>
__device__ __forceinline__ void discard_partials(const TC* C, int64_t stride, int ns, int64_t b0,
                                                 int64_t e0) {
  for (int k = threadIdx.x & 31; k < ns; k += 32) {
    const uintptr_t lo = reinterpret_cast<uintptr_t>(C + k * stride + b0);
    const uintptr_t hi = reinterpret_cast<uintptr_t>(C + k * stride + e0);
    for (uintptr_t a = (lo + 127) & ~uintptr_t(127); a + 128 <= hi; a += 128)
      asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
  }
}

static int vec_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > kRedMaxBlocks) b = kRedMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

// One output element t of the epilogue (acc: this thread's share of the
// reduction of its mode).
template <typename TC, typename TO>
__device__ __forceinline__ void combine_elem(int mode, const TC* __restrict__ C,
                                             int64_t split_stride, int nsplit, int n, int64_t t,
                                             const double* __restrict__ dK,
                                             const double* __restrict__ V,
                                             const double* __restrict__ Bv, TO* __restrict__ out,
                                             double lam, double rho, double (&acc)[1]) {
  // the split partials in order; loaded eight at a time so that their
  // latencies overlap (the sum is the same, term by term)
  double c = 0.0;
  int k = 0;
  for (; k + 8 <= nsplit; k += 8) {
    TC v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = C[(k + u) * split_stride + t];
#pragma unroll
    for (int u = 0; u < 8; ++u) c += (double)v[u];
  }
  for (; k < nsplit; ++k) c += (double)C[k * split_stride + t];
  const int i = (int)(t % n);
  double o;
  if (mode == CM_STORE) {
    o = c;
  } else if (mode == CM_DK || mode == CM_DK_NORM) {
    o = dK[i] * c;
    acc[0] += o * o;
  } else {
    const double y = dK[i] * c + (lam * dK[i] + rho) * V[t];
    if (mode == CM_APPLY) {
      o = y;
      acc[0] += V[t] * y;
    } else {
      o = Bv[t] - y;
      acc[0] += o * o;
    }
  }
  out[t] = (TO)o;
}

template <typename TC, typename TO>
__global__ void __launch_bounds__(256)
combine_kernel(int mode, const TC* __restrict__ C, int64_t split_stride, int nsplit, int n, int r,
               const double* __restrict__ dK, const double* __restrict__ V,
               const double* __restrict__ Bv, TO* __restrict__ out, DevScalars* s,
               RedScratch red, const DevScalars* skip) {
  if (mode != CM_RESID && mode != CM_TRUE && dev_skip(skip)) return;
  const int64_t total = (int64_t)n * r;
  double lam = 0.0, rho = 0.0;
  if (s) { lam = s->lam; rho = s->rho; }
  double acc[1] = {0.0};
  // warp-uniform loop (blockDim is a multiple of 32): lane l takes t = t0 + l
  const int lane = threadIdx.x & 31;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane; t0 < total;
       t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + lane;
    if (t < total)
      combine_elem<TC, TO>(mode, C, split_stride, nsplit, n, t, dK, V, Bv, out, lam, rho, acc);
    __syncwarp();
    discard_partials(C, split_stride, nsplit, t0, t0 + 32 < total ? t0 + 32 : total);
  }
  if (mode == CM_APPLY || mode == CM_RESID || mode == CM_TRUE || mode == CM_DK_NORM) {
    double tot[1];
    if (grid_sum_last<1>(acc, red, tot)) {
      if (mode == CM_DK_NORM) {
        s->bb = tot[0];
      } else if (mode == CM_APPLY) {
        s->pAp = tot[0];
        const double a = s->rz / tot[0];
        if (!(tot[0] > 0.0) || !isfinite(a)) {
          s->status = 5;  // CPHIFI_E_BREAKDOWN
          s->done = 1;
        }
        s->alpha = a;
      } else {
        s->true_rr = tot[0];
        if (mode == CM_RESID) {
          s->rr = tot[0];
          s->inner_done = 0;
        }
        s->true_evals += 1;
        if (!isfinite(tot[0])) { s->status = 5; s->done = 1; }
        else if (s->status == 0) s->done = (tot[0] <= s->tol2 * s->bb) ? 1 : 0;
      }
    }
  }
}

__global__ void adopt_residual_kernel(const double* __restrict__ tres, double* __restrict__ res,
                                      int64_t count, DevScalars* s) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    res[t] = tres[t];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s->rr = s->true_rr;
    s->inner_done = 0;
  }
}

cudaError_t launch_adopt_residual(const double* tres, double* res, int64_t count, DevScalars* s,
                                  cudaStream_t st) {
  adopt_residual_kernel<<<vec_blocks(count), 256, 0, st>>>(tres, res, count, s);
  return cudaGetLastError();
}

template <typename TC, typename TO>
cudaError_t launch_combine(int mode, const TC* C, int64_t split_stride, int nsplit, int n, int r,
                           const double* dK, const double* V, const double* Bv, TO* out,
                           DevScalars* s, RedScratch red, const DevScalars* skip,
                           cudaStream_t st) {
  const int blocks = vec_blocks((int64_t)n * r);
  combine_kernel<TC, TO><<<blocks, 256, 0, st>>>(mode, C, split_stride, nsplit, n, r, dK, V, Bv,
                                                 out, s, red, skip);
  return cudaGetLastError();
}

template cudaError_t launch_combine<double, double>(int, const double*, int64_t, int, int, int,
                                                    const double*, const double*, const double*,
                                                    double*, DevScalars*, RedScratch, const DevScalars*,
                                                    cudaStream_t);
template cudaError_t launch_combine<float, float>(int, const float*, int64_t, int, int, int,
                                                  const double*, const double*, const double*,
                                                  float*, DevScalars*, RedScratch, const DevScalars*,
                                                  cudaStream_t);
template cudaError_t launch_combine<double, float>(int, const double*, int64_t, int, int, int,
                                                   const double*, const double*, const double*,
                                                   float*, DevScalars*, RedScratch, const DevScalars*,
                                                   cudaStream_t);
template cudaError_t launch_combine<float, double>(int, const float*, int64_t, int, int, int,
                                                   const double*, const double*, const double*,
                                                   double*, DevScalars*, RedScratch, const DevScalars*,
                                                   cudaStream_t);

// --------------------------------- update + preconditioner (Eq. fx) --------
// A block walks tiles of kUpRows kernel-eigenbasis rows.  UP_ITER first applies
// x += alpha p, r -= alpha y (FP64).  Then, per row i,
// z(i,:) = ((r(i,:) U_V) .* D(i,:)) U_V' as two small products through
// shared memory in arithmetic TP, and the last block turns (r, z) and ||r||^2
// into beta and the convergence flags.
// Tiles of 64 rows; 16 when the rows would otherwise occupy fewer blocks
// than there are SMs (small n: more blocks share the r x r products).
template <typename TP, int kUpRows>
__global__ void __launch_bounds__(256)
update_precond_kernel(int mode, int n, int r, double* __restrict__ x, double* __restrict__ rres,
                      const double* __restrict__ p, const double* __restrict__ y,
                      double* __restrict__ z, const TP* __restrict__ UV,
                      const TP* __restrict__ D, DevScalars* s, RedScratch red) {
  if (mode == UP_ITER ? dev_skip(s) : s->done) return;
  extern __shared__ unsigned char up_smem[];
  TP* uv = (TP*)up_smem;                    // r x r, U_V(j, k) at j + r k
  TP* Rt = uv + r * r;                      // kUpRows x (r + 1)
  TP* Tt = Rt + kUpRows * (r + 1);          // kUpRows x (r + 1)
  const int ld = r + 1;
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) uv[t] = UV[t];
  const double alpha = mode == UP_ITER ? s->alpha : 0.0;
  double acc[2] = {0.0, 0.0};  // (r, z), ||r||^2
  const int ntiles = (n + kUpRows - 1) / kUpRows;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = tile * kUpRows;
    const int rows = min(kUpRows, n - i0);
    __syncthreads();
    for (int e = threadIdx.x; e < kUpRows * r; e += blockDim.x) {
      const int il = e % kUpRows, j = e / kUpRows;
      if (il >= rows) continue;
      const int64_t t = (int64_t)j * n + i0 + il;
      double rj = rres[t];
      if (mode == UP_ITER) {
        x[t] += alpha * p[t];
        rj -= alpha * y[t];
        rres[t] = rj;
      }
      acc[1] += rj * rj;
      Rt[il * ld + j] = (TP)rj;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kUpRows * r; e += blockDim.x) {
      const int il = e % kUpRows, k = e / kUpRows;
      if (il >= rows) continue;
      TP a = TP(0);
      for (int j = 0; j < r; ++j) a += Rt[il * ld + j] * uv[j + r * k];
      Tt[il * ld + k] = a * D[(int64_t)k * n + i0 + il];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kUpRows * r; e += blockDim.x) {
      const int il = e % kUpRows, j = e / kUpRows;
      if (il >= rows) continue;
      TP a = TP(0);
      for (int k = 0; k < r; ++k) a += Tt[il * ld + k] * uv[j + r * k];
      const int64_t t = (int64_t)j * n + i0 + il;
      z[t] = (double)a;
      acc[0] += rres[t] * (double)a;
    }
  }
  double tot[2];
  if (grid_sum_last<2>(acc, red, tot)) {
    const double rz_new = tot[0];
    s->rr = tot[1];
    if (mode == UP_ITER) {
      s->iter += 1;
      s->beta = rz_new / s->rz;
      if (!isfinite(s->beta) || !isfinite(tot[1])) { s->status = 5; s->done = 1; }
      if (tot[1] <= s->tol2 * s->bb) {
        if (s->mode == 0) s->done = 1; else s->inner_done = 1;
      }
      if (s->iter >= s->max_iter) s->inner_done = 1;
    } else {
      s->beta = 0.0;
      s->restarts += 1;
      if (!isfinite(rz_new)) { s->status = 5; s->done = 1; }
    }
    s->rz = rz_new;
  }
}

template <typename TP>
cudaError_t launch_update_precond(int mode, int n, int r, double* x, double* rres,
                                  const double* p, const double* y, double* z, const TP* UV,
                                  const TP* D, DevScalars* s, RedScratch red, cudaStream_t st) {
  if (r < 1 || r > kMaxRank) return cudaErrorInvalidValue;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool narrow = (n + 63) / 64 < sms;
  const int rows = narrow ? 16 : 64;
  int blocks = (n + rows - 1) / rows;
  if (blocks > kRedMaxBlocks) blocks = kRedMaxBlocks;
  if (blocks < 1) blocks = 1;
  const size_t smem = (size_t)(r * r + 2 * rows * (r + 1)) * sizeof(TP);
  auto kern = narrow ? update_precond_kernel<TP, 16> : update_precond_kernel<TP, 64>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<blocks, 256, smem, st>>>(mode, n, r, x, rres, p, y, z, UV, D, s, red);
  return cudaGetLastError();
}

template cudaError_t launch_update_precond<double>(int, int, int, double*, double*, const double*,
                                                   const double*, double*, const double*,
                                                   const double*, DevScalars*, RedScratch,
                                                   cudaStream_t);
template cudaError_t launch_update_precond<float>(int, int, int, double*, double*, const double*,
                                                  const double*, double*, const float*,
                                                  const float*, DevScalars*, RedScratch,
                                                  cudaStream_t);

// -------------------------------------------------- direction update ------
// p = z + beta p, and the operand of the next product in the low-precision
// types: pop = TB(scale[i] p(i, j)) (the D_K row scale of the eigenbasis
// operator folded in; scale may be NULL) with leading dimension ldp, and the
// same in BF16 when pop16 is set.
template <typename TB>
__global__ void pupdate_kernel(int n, int r, const double* __restrict__ z, double* __restrict__ p,
                               TB* __restrict__ pop, const double* __restrict__ scale,
                               int64_t ldp, __nv_bfloat16* __restrict__ pop16, DevScalars* s) {
  if (dev_skip(s)) return;
  const double beta = s->beta;
  const int64_t total = (int64_t)n * r;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    // beta = 0 (a restart): p = z without reading p, which a new solve finds
    // holding whatever its memory held before (0 * NaN would be NaN)
    const double v = beta != 0.0 ? z[t] + beta * p[t] : z[t];
    p[t] = v;
    const int64_t i = t % n, j = t / n;
    const double sv = scale ? scale[i] * v : v;
    if (pop) pop[j * ldp + i] = (TB)sv;
    if (pop16) pop16[j * ldp + i] = __double2bfloat16(sv);
  }
}

template <typename TB>
cudaError_t launch_pupdate(int n, int r, const double* z, double* p, TB* pop, const double* scale,
                           int64_t ldp, __nv_bfloat16* pop16, DevScalars* s, cudaStream_t st) {
  const int blocks = vec_blocks((int64_t)n * r);
  pupdate_kernel<TB><<<blocks, 256, 0, st>>>(n, r, z, p, pop, scale, ldp, pop16, s);
  return cudaGetLastError();
}

template cudaError_t launch_pupdate<double>(int, int, const double*, double*, double*,
                                            const double*, int64_t, __nv_bfloat16*, DevScalars*,
                                            cudaStream_t);
template cudaError_t launch_pupdate<float>(int, int, const double*, double*, float*, const double*,
                                           int64_t, __nv_bfloat16*, DevScalars*, cudaStream_t);

// ---------------------------------------------------- small utilities -----
// Y(i,:) = ((X(i,:) U_V) .* D(i,:)) U_V' (the r x r part of Eq. fx), FP64.
__global__ void precond_only_kernel(int n, int r, const double* __restrict__ X,
                                    double* __restrict__ Y, const double* __restrict__ UV,
                                    const double* __restrict__ D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t[kMaxRank];
  for (int k = 0; k < r; ++k) {
    double a = 0.0;
    for (int j = 0; j < r; ++j) a += X[(int64_t)j * n + i] * UV[j + r * k];
    t[k] = a * D[(int64_t)k * n + i];
  }
  for (int j = 0; j < r; ++j) {
    double a = 0.0;
    for (int k = 0; k < r; ++k) a += t[k] * UV[j + r * k];
    Y[(int64_t)j * n + i] = a;
  }
}

cudaError_t launch_precond_only(int n, int r, const double* X, double* Y, const double* UV,
                                const double* D, cudaStream_t st) {
  precond_only_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, r, X, Y, UV, D);
  return cudaGetLastError();
}

template <typename TS, typename TD>
__global__ void convert_kernel(const TS* __restrict__ a, TD* __restrict__ b, int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    b[t] = (TD)a[t];
}

template <typename TS, typename TD>
cudaError_t launch_convert(const TS* src, TD* dst, int64_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int blocks = (int)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096);
  convert_kernel<TS, TD><<<blocks, 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

}  // namespace cphifi
