// Symmetric eigendecomposition K = U_K diag(D_K) U_K' in FP64 on the device
// (Eq. eigK, §3.2: the one-time setup of a kernel matrix), by the cyclic
// two-sided Jacobi method with a parallel ordering.
//
// Each sweep visits every index pair (p, q) once, in m - 1 rounds of m/2
// disjoint pairs (m = n rounded up to even; the round-robin "circle" schedule,
// a pair with the padding index m - 1 >= n is skipped).  For each pair of a
// round the 2 x 2 symmetric Schur rotation (c, s) that zeroes a_pq is formed
// (Golub & Van Loan, Matrix Computations, 4th ed., §8.5.2); the round then
// applies all of them at once: A <- A J and V <- V J (the columns p, q of each
// pair: one block per pair), then A <- J' A (each column j of A is read into
// shared memory, its rows p, q rotated for every pair, and written back: one
// block per column), so both passes read and write whole columns, coalesced.
// A is kept in its own columns; V accumulates the rotations, so that at the
// end A = V' K V is diagonal to FP64 round-off, D_K = diag(A), U_K = V.
// A rotation is skipped when |a_pq| <= max(1e-18 ||K||_F, 4 eps sqrt(|a_pp
// a_qq|)) (the relative test of Demmel and Veselic, with an absolute floor);
// the sweeps stop after one that applied no rotation.  The rounds of one
// sweep are one CUDA graph, replayed sweep after sweep.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "cphifi.h"
#include "launch.h"

namespace cphifi {
namespace {

struct Rot {
  int p, q;
  double c, s;
  double app, aqq;  // the new diagonal entries a_pp - t a_pq, a_qq + t a_pq
};

// Pair t of round k of the circle schedule on m (even) indices: index m-1 is
// fixed, the others sit on a circle of m-1; i0 = k/2 (mod m-1) meets m-1 and
// i0 + t meets i0 - t.  Over the m-1 rounds every pair meets exactly once.
__device__ __forceinline__ void round_pair(int k, int t, int m, int* p, int* q) {
  const int h = m - 1;
  const int i0 = (int)(((int64_t)k * (m / 2)) % h);
  if (t == 0) {
    *p = i0;
    *q = m - 1;
  } else {
    *p = (i0 + t) % h;
    *q = (i0 - t + h) % h;
  }
}

// One block per pair: the rotation from the current a_pp, a_qq, a_pq (only
// this block touches columns p and q in this pass), then A <- A J and
// V <- V J on those two columns.
__global__ void __launch_bounds__(256) jacobi_cols_kernel(double* __restrict__ A,
                                                          double* __restrict__ V, int n, int m,
                                                          int k, double skip_abs,
                                                          Rot* __restrict__ rot,
                                                          int* __restrict__ slot,
                                                          unsigned* __restrict__ nrot) {
  const int t = blockIdx.x;
  int p, q;
  round_pair(k, t, m, &p, &q);
  __shared__ double cs[2];
  if (threadIdx.x == 0) {
    double c = 1.0, s = 0.0, app = 0.0, aqq = 0.0;
    if (p < n) slot[p] = t;
    if (q < n) slot[q] = t;
    if (p < n && q < n) {
      app = A[p + (int64_t)p * n];
      aqq = A[q + (int64_t)q * n];
      const double apq = 0.5 * (A[p + (int64_t)q * n] + A[q + (int64_t)p * n]);
      if (fabs(apq) > fmax(skip_abs, 8.9e-16 * sqrt(fabs(app) * fabs(aqq)))) {
        atomicAdd(nrot, 1u);
        const double tau = (aqq - app) / (2.0 * apq);
        const double tt = fabs(tau) > 1e150
                              ? 0.5 / tau
                              : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + tt * tt);
        s = tt * c;
        app -= tt * apq;
        aqq += tt * apq;
      }
    }
    rot[t] = Rot{p, q, c, s, app, aqq};
    cs[0] = c;
    cs[1] = s;
  }
  __syncthreads();
  if (p >= n || q >= n) return;
  const double c = cs[0], s = cs[1];
  if (s == 0.0) return;
  double* ap = A + (int64_t)p * n;
  double* aq = A + (int64_t)q * n;
  double* vp = V + (int64_t)p * n;
  double* vq = V + (int64_t)q * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = ap[i], y = aq[i];
    ap[i] = c * x - s * y;
    aq[i] = s * x + c * y;
    const double u = vp[i], w = vq[i];
    vp[i] = c * u - s * w;
    vq[i] = s * u + c * w;
  }
}

// One block per column j (grid-stride): A <- J' A on column j, i.e. rows p, q
// of every pair; then the entries the rotation of j's own pair set exactly:
// the new diagonal entry and the zeroed off-diagonal one.
__global__ void __launch_bounds__(256) jacobi_rows_kernel(double* __restrict__ A, int n,
                                                          int npairs,
                                                          const Rot* __restrict__ rot,
                                                          const int* __restrict__ slot) {
  extern __shared__ double col[];
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    double* a = A + (int64_t)j * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = a[i];
    __syncthreads();
    for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
      const Rot R = rot[t];
      if (R.p >= n || R.q >= n || R.s == 0.0) continue;
      const double x = col[R.p], y = col[R.q];
      col[R.p] = R.c * x - R.s * y;
      col[R.q] = R.s * x + R.c * y;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const Rot R = rot[slot[j]];  // j's own pair in this round
      if (R.p < n && R.q < n && R.s != 0.0) {
        col[j] = R.p == j ? R.app : R.aqq;
        col[R.p == j ? R.q : R.p] = 0.0;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = col[i];
    __syncthreads();
  }
}

// out[0] = sum of squares off the diagonal, out[1] = on it (one block).
__global__ void __launch_bounds__(1024) jacobi_offdiag_kernel(const double* __restrict__ A, int n,
                                                              double* out) {
  __shared__ double sm[64];
  double v[2] = {0.0, 0.0};
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
    const double x = A[e];
    const int64_t i = e % n, j = e / n;
    if (i == j) v[1] += x * x; else v[0] += x * x;
  }
  block_sum<2>(v, sm);
  if (threadIdx.x == 0) {
    out[0] = v[0];
    out[1] = v[1];
  }
}

// Column gather U(:, k) = V(:, perm[k]).
__global__ void gather_cols_kernel(const double* __restrict__ V, const int* __restrict__ perm,
                                   int n, double* __restrict__ U) {
  const int k = blockIdx.y;
  const double* src = V + (int64_t)perm[k] * n;
  double* dst = U + (int64_t)k * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void identity_kernel(double* V, int n) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x)
    V[e] = (e % n == e / n) ? 1.0 : 0.0;
}

// Mirror the lower triangle into the upper one (the lower triangle is read).
__global__ void symmetrize_lower_kernel(double* A, int n) {
  const int64_t nn = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    if (i < j) A[e] = A[j + i * n];
  }
}

}  // namespace

int sym_eig_max_n() { return kSymEigMaxN; }

// A (n x n, column-major, lower triangle read) is overwritten by the
// eigenvectors (columns, eigenvalues ascending); w gets the eigenvalues.
// Synchronous on `st`.  Returns CPHIFI_OK, CPHIFI_E_OOM, CPHIFI_E_DEVICE or
// CPHIFI_E_INVALID_ARG (no convergence within the sweep limit).
int sym_eig_jacobi(double* A, int n, double* w, cudaStream_t st, std::string* why) {
  if (n < 1 || n > kSymEigMaxN) {
    *why = "n outside the device eigensolver's range";
    return CPHIFI_E_UNSUPPORTED;
  }
  const int m = n + (n & 1);
  const int npairs = m / 2;
  const size_t nn = (size_t)n * n;
  double* V = nullptr;
  Rot* rot = nullptr;
  int* slot = nullptr;
  unsigned* nrot = nullptr;
  double* red = nullptr;
  int* perm_d = nullptr;
  double* hred = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = CPHIFI_OK;
  auto done = [&](int code, const char* msg) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFree(V);
    cudaFree(rot);
    cudaFree(slot);
    cudaFree(nrot);
    cudaFree(red);
    cudaFree(perm_d);
    if (hred) cudaFreeHost(hred);
    if (code != CPHIFI_OK) {
      cudaGetLastError();
      *why = msg;
    }
    return code;
  };
  if (cudaMalloc(&V, nn * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&rot, (size_t)npairs * sizeof(Rot)) != cudaSuccess ||
      cudaMalloc(&slot, (size_t)m * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&nrot, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&red, 2 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&perm_d, (size_t)n * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&hred, 2 * sizeof(double)) != cudaSuccess)
    return done(CPHIFI_E_OOM, "workspace allocation for the eigensolver failed");
  const size_t smem = (size_t)n * sizeof(double);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(jacobi_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return done(CPHIFI_E_DEVICE, "eigensolver: shared-memory attribute");
  const int eb = (int)std::min<size_t>((nn + 255) / 256, 4096);
  symmetrize_lower_kernel<<<eb, 256, 0, st>>>(A, n);
  identity_kernel<<<eb, 256, 0, st>>>(V, n);
  jacobi_offdiag_kernel<<<1, 1024, 0, st>>>(A, n, red);
  if (cudaMemcpyAsync(hred, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return done(CPHIFI_E_DEVICE, "eigensolver: setup kernels failed");
  const double total = hred[0] + hred[1];
  // rotations whose a_pq is below this are skipped (they cannot change A at
  // FP64 precision relative to its norm)
  const double skip_abs = 1e-18 * std::sqrt(total);
  const int rows_grid = std::min(n, 1024);
  unsigned* hrot = reinterpret_cast<unsigned*>(hred);  // (red's pinned copy is free now)
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return done(CPHIFI_E_DEVICE, "eigensolver: graph capture");
  cudaMemsetAsync(nrot, 0, sizeof(unsigned), st);
  for (int k = 0; k < m - 1; ++k) {
    jacobi_cols_kernel<<<npairs, 256, 0, st>>>(A, V, n, m, k, skip_abs, rot, slot, nrot);
    jacobi_rows_kernel<<<rows_grid, 256, smem, st>>>(A, n, npairs, rot, slot);
  }
  cudaMemcpyAsync(hrot, nrot, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  if (ec != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
    return done(CPHIFI_E_DEVICE, "eigensolver: graph instantiation");
  bool converged = total == 0.0;
  for (int sweep = 0; sweep < kSymEigMaxSweeps && !converged; ++sweep) {
    if (cudaGraphLaunch(exec, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return done(CPHIFI_E_DEVICE, "eigensolver: sweep failed");
    converged = *hrot == 0u;
  }
  if (!converged) rc = CPHIFI_E_INVALID_ARG;
  // eigenvalues ascending, eigenvectors in the same order
  std::vector<double> d(n);
  if (cudaMemcpy2DAsync(d.data(), sizeof(double), A, (size_t)(n + 1) * sizeof(double),
                        sizeof(double), n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return done(CPHIFI_E_DEVICE, "eigensolver: reading the eigenvalues");
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return d[a] < d[b]; });
  std::vector<double> ds(n);
  for (int k = 0; k < n; ++k) ds[k] = d[perm[k]];
  if (cudaMemcpyAsync(perm_d, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(w, ds.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return done(CPHIFI_E_DEVICE, "eigensolver: writing the eigenvalues");
  gather_cols_kernel<<<dim3((n + 255) / 256 < 8 ? (n + 255) / 256 : 8, n), 256, 0, st>>>(
      V, perm_d, n, A);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return done(CPHIFI_E_DEVICE, "eigensolver: ordering the eigenvectors");
  return done(rc, "the eigensolver did not converge within the sweep limit");
}

}  // namespace cphifi
