// Shared device-side definitions of the GB300 kernel-mode PCG solver.
//
// Layout used by every kernel: n x r matrices are column-major with leading
// dimension n (vec order of the paper: element (i, j) at i + n*j).  The
// observation-indexed matrix Zhat (Eq. zhat, §4.2) is stored the same way,
// q x r column-major ("structure of arrays"): Zhat(l, j) at j*zld + l, so a
// warp reading 32 consecutive observations of one column issues one 128-byte
// (FP32) or 256-byte (FP64) coalesced load.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cphifi {

constexpr int kMaxRank = 64;
constexpr int kRedMaxBlocks = 1024;  // capacity of the reduction partial buffer
constexpr int kRedSlots = 4;         // doubles per block in that buffer

// Scalars of one PCG run.  They live in device memory so that the
// iteration never needs the host: every kernel reads the step sizes it needs
// and the last block of each reduction writes the next ones.
struct DevScalars {
  double rz;        // (r, z) of the current residual
  double rz_new;
  double pAp;       // (p, A p)
  double alpha;
  double beta;
  double rr;        // ||r||^2 of the recurrence residual
  double bb;        // ||b||^2
  double tol2;      // tol^2
  double true_rr;   // ||b - A x||^2 at the last FP64 true residual
  double lam;       // lambda of this solve
  double rho;       // rho of this solve
  int iter;         // operator applications inside the PCG loop
  int max_iter;
  int inner_done;   // recurrence residual reached tol (or max_iter) in this cycle
  int done;         // the solve is finished: skip every remaining kernel
  int status;       // 0, or CPHIFI_E_BREAKDOWN
  int true_evals;
  int restarts;
  int mode;         // 0: FP64 (stop on the recurrence); 1: mixed (stop on true residual)
};

struct RedScratch {
  double* partials;    // kRedMaxBlocks * kRedSlots
  unsigned* ticket;    // zero between kernels
};

__device__ __forceinline__ bool dev_skip(const DevScalars* s) {
  // A solve that finished, or an inner cycle that converged, turns the rest
  // of the launched kernels into no-ops.
  return s != nullptr && (s->done | s->inner_done);
}

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// Deterministic block sum of NV doubles; the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm /* NV*32 */) {
  warp_sum<NV>(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k * 32 + w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = lane < nw ? sm[k * 32 + lane] : 0.0;
    warp_sum<NV>(v);
  }
}

// Grid-wide deterministic sum: each block writes its partial, the last block
// to arrive (ticket) adds the partials in block order and returns true in
// thread 0 with the totals in `tot`.  Every thread of every block must call it.
template <int NV>
__device__ bool grid_sum_last(double (&v)[NV], RedScratch red, double (&tot)[NV]) {
  __shared__ double sm[NV * 32];
  __shared__ int is_last;
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red.partials[blockIdx.x * kRedSlots + k] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(red.ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&red.partials[b * kRedSlots + k]);
  block_sum<NV>(acc, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = acc[k];
    *red.ticket = 0u;
  }
  return threadIdx.x == 0;
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

}  // namespace cphifi
