// Many independent kernel-mode PCG solves (§4.4, mixed precision: FP32
// operator, FP64 scalars, FP64-accurate true residual every k iterations) in
// one persistent launch.
//
// A request's solve is a chain of phases; a phase is a set of tiles that do
// not depend on one another:
//   set-up        D (Eq. fx's diagonal) and x = 0                 vector tiles
//   rhs product   U_K' B, double-float, k-split partials          product tiles
//   rhs combine   bbar = D_K U_K' B, r = bbar, ||bbar||^2         vector tiles
//   restart       z = M^-1 r (Eq. fx), (r, z), ||r||^2             vector tiles
//   product 1     p = z + beta p (stored by the first row block),
//                 Xhat = U_K fl32(D_K p), FP32 partials            product tiles
//   gather        Yhat1 from Xhat (Eqs. vl, yhat1), FP32           8 virtual warps each
//   product 2     U_K' Yhat1, FP32 partials                        product tiles
//   combine       y = D_K U_K' Yhat1 + (lambda D_K + rho) p, (p, y) vector tiles
//   update        x += alpha p, r -= alpha y, z = M^-1 r            vector tiles
//   true residual the operator on x in double-float (products, gather), then
//                 b - A x and its norm (four phases)
//   final         W = U_K x, double-float (two phases)
// Tiles that produce sums store one partial per tile; the block that
// finishes the last tile of a phase adds them in tile order, takes the PCG's
// decisions (alpha, beta, convergence on the recurrence or on the true
// residual, restart from the true residual, max_iter) exactly as the
// step-by-step path does, and opens the next phase.  Results therefore do
// not depend on which block ran which tile, nor on the other requests of the
// launch.
//
// Scheduling: a request's claim word holds its open phase, that phase's tile
// count and the tiles claimed so far.  A block looking for work reads the
// claim words (one per thread), takes the first request in the given order
// that has an unclaimed tile and claims with an atomic add on that word; the
// claim is valid when the returned count is below the returned tile count,
// and the returned word names the phase (the phase cannot change until that
// tile is done).  Data written by other blocks in this launch is read through
// L2 (__ldcg / volatile), never through the non-coherent L1.  No tile waits
// for another; idle blocks poll with a growing sleep and give up when no
// tile has finished anywhere for timeout_ns (BatchCtl::err = 1, every block
// leaves).
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "cphifi.h"
#include "df.cuh"
#include "gds.cuh"
#include "launch.h"

namespace cphifi {
namespace {

enum : int {
  BP_SETUP = 0,
  BP_RHS_PROD,
  BP_RHS_COMB,
  BP_RESTART,
  BP_PROD1,
  BP_GDS,
  BP_PROD2,
  BP_COMB2,
  BP_UPDATE,
  BP_TR_PROD1,
  BP_TR_GDS,
  BP_TR_PROD2,
  BP_TR_COMB,
  BP_FINAL_PROD,
  BP_FINAL_COMB,
  BP_DONE
};
static_assert(BP_DONE == kBatchPhaseDone, "phase numbering");

#ifndef CPHIFI_BATCH_SLEEP_MAX_NS
#define CPHIFI_BATCH_SLEEP_MAX_NS 1024
#endif
constexpr int kThreads = 256;
constexpr unsigned kSleepMaxNs = CPHIFI_BATCH_SLEEP_MAX_NS;  // longest idle sleep
constexpr int kBK32 = 16;  // k slab of the FP32 product tile
constexpr int kBKdf = 16;  // k slab of the double-float product tile

__host__ __device__ inline int vec_tiles(const BatchReq& q) {
  return (q.n + kBatchRows - 1) / kBatchRows;
}
__host__ __device__ inline int row_blocks(const BatchReq& q) {
  return (q.n + kBatchBM - 1) / kBatchBM;
}
__host__ __device__ inline int row_blocks_df(const BatchReq& q) {
  return (q.n + kBatchBMdf - 1) / kBatchBMdf;
}
__host__ __device__ inline int phase_tiles(const BatchReq& q, int ph) {
  switch (ph) {
    case BP_RHS_PROD:
    case BP_TR_PROD1:
    case BP_TR_PROD2:
    case BP_FINAL_PROD:
      return row_blocks_df(q) * q.sdf;
    case BP_PROD1:
    case BP_PROD2:
      return row_blocks(q) * q.s32;
    case BP_GDS:
    case BP_TR_GDS:
      return (q.pl.nwarps + 7) / 8;
    case BP_DONE:
      return 0;
    default:
      return vec_tiles(q);
  }
}

// Claim word: tiles of the open phase (20 bits) | phase (5) | aux (3) |
// 4 unused | tiles claimed (32), aux = adopt (bit 0: the restart starts
// from the true residual) | par << 1 (which of the two p buffers is the
// current direction).  A claim's atomic add returns all a block needs to run
// its tile.
__host__ __device__ inline unsigned long long claim_word(int tiles, int phase, int aux) {
  return ((unsigned long long)tiles << 44) | ((unsigned long long)phase << 39) |
         ((unsigned long long)(aux & 7) << 36);
}
__device__ __forceinline__ unsigned claim_count(unsigned long long w) { return (unsigned)w; }
__device__ __forceinline__ int claim_tiles(unsigned long long w) { return (int)(w >> 44); }
__device__ __forceinline__ int claim_phase(unsigned long long w) { return (int)(w >> 39) & 31; }
__device__ __forceinline__ int claim_aux(unsigned long long w) { return (int)(w >> 36) & 7; }

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The claiming block's copy (shared memory) of what a tile and the phase's
// decisions read: the request's descriptor, its scalars and its state.  The
// scalars and the state change only in the decisions that close a phase, so
// the copy taken at a claim holds for the whole phase; the block that takes
// the decisions updates its copy as it writes them back.
struct BatchLocal {
  BatchReq q;
  DevScalars s;
  int chunk, adopt, par, iters;
};

// ---------------------------------------------------------- vector tiles --
// Rows [32 t, 32 t + 32) of the n x r arrays, all r columns; 256 threads
// walk the 32 r elements (32 consecutive rows of one column per warp: one
// coalesced segment).  Partial sums go to red[2 t], red[2 t + 1].
constexpr int kVecPerThread = kBatchRows * kMaxRank / kThreads;  // 8

// The restart and update phases: the rows of r (from the true residual on an
// adopting restart, or after x += alpha p, r -= alpha y) and
// z = ((r U_V) .* D) U_V' (Eq. fx in the eigenbasis, FP32 as in the mixed
// solve), with (r, z) and ||r||^2.
__device__ __forceinline__ void precond_tile(int ph, const BatchReq& q, const DevScalars& ss,
                                             int aux, int tile, float* sm, double (&acc)[2]) {
  const int adopt = aux & 1;
  const double* pc = q.p[(aux >> 1) & 1];  // the current direction
  const int n = q.n, r = q.r, ld = r + 1;
  float* uv = sm;                        // r x r, U_V(j, k) at j + r k
  float* Rt = uv + r * r;                // 32 x (r + 1)
  float* Tt = Rt + kBatchRows * ld;      // 32 x (r + 1)
  const int i0 = tile * kBatchRows;
  const int rows = min(kBatchRows, n - i0);
  for (int t = threadIdx.x; t < r * r; t += kThreads) uv[t] = q.UV32[t];
  const double alpha = ph == BP_UPDATE ? ss.alpha : 0.0;
  double rv[kVecPerThread];
#pragma unroll
  for (int u = 0; u < kVecPerThread; ++u) {
    const int e = threadIdx.x + kThreads * u;
    rv[u] = 0.0;
    if (e >= kBatchRows * r) continue;
    const int il = e % kBatchRows, j = e / kBatchRows;
    double rj = 0.0;
    if (il < rows) {
      const int64_t t = (int64_t)j * n + i0 + il;
      if (ph == BP_UPDATE) {
        q.x[t] = __ldcg(q.x + t) + alpha * __ldcg(pc + t);
        rj = __ldcg(q.res + t) - alpha * __ldcg(q.y + t);
        q.res[t] = rj;
      } else if (adopt) {
        rj = __ldcg(q.tres + t);
        q.res[t] = rj;
      } else {
        rj = __ldcg(q.res + t);
      }
      acc[1] += rj * rj;
    }
    rv[u] = rj;
    Rt[il * ld + j] = (float)rj;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kBatchRows * r; e += kThreads) {
    const int il = e % kBatchRows, k = e / kBatchRows;
    if (il >= rows) continue;
    float a = 0.f;
    for (int j = 0; j < r; ++j) a += Rt[il * ld + j] * uv[j + r * k];
    Tt[il * ld + k] = a * __ldcg(q.D32 + (int64_t)k * n + i0 + il);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kVecPerThread; ++u) {
    const int e = threadIdx.x + kThreads * u;
    if (e >= kBatchRows * r) continue;
    const int il = e % kBatchRows, j = e / kBatchRows;
    if (il >= rows) continue;
    float a = 0.f;
    for (int k = 0; k < r; ++k) a += Tt[il * ld + k] * uv[j + r * k];
    q.z[(int64_t)j * n + i0 + il] = (double)a;
    acc[0] += rv[u] * (double)a;
  }
}

__device__ __noinline__ void vec_tile(int ph, const BatchReq& q, const DevScalars& ss, int aux,
                                      int tile, unsigned char* smem, double* sred) {
  const int n = q.n, r = q.r;
  const int64_t nr = (int64_t)n * r;
  const int i0 = tile * kBatchRows;
  const int rows = min(kBatchRows, n - i0);
  double acc[2] = {0.0, 0.0};
  if (ph == BP_RESTART || ph == BP_UPDATE) {
    precond_tile(ph, q, ss, aux, tile, reinterpret_cast<float*>(smem), acc);
  } else {
    const double* pc = q.p[(aux >> 1) & 1];
    for (int e = threadIdx.x; e < kBatchRows * r; e += kThreads) {
      const int il = e % kBatchRows, j = e / kBatchRows;
      if (il >= rows) continue;
      const int i = i0 + il;
      const int64_t t = (int64_t)j * n + i;
      switch (ph) {
        case BP_SETUP: {
          // D(i, j) = 1 / (gamma D_V(j) D_K(i)^2 + lambda D_K(i) + rho), round-off
          // negative eigenvalues of the PSD K and V clamped to 0
          const double k = fmax(q.dK[i], 0.0), v = fmax(q.dV[j], 0.0);
          const double d = 1.0 / (q.gamma * v * k * k + q.lam * k + q.rho);
          q.D64[t] = d;
          q.D32[t] = (float)d;
          q.x[t] = 0.0;
          break;
        }
        case BP_RHS_COMB: {
          double c = 0.0;
          for (int s = 0; s < q.sdf; ++s) c += __ldcg(q.cpd + s * nr + t);
          const double o = q.dK[i] * c;
          q.bbar[t] = o;
          q.res[t] = o;
          acc[0] += o * o;
          break;
        }
        case BP_COMB2: {
          double c = 0.0;
          for (int s = 0; s < q.s32; ++s) c += (double)__ldcg(q.cp32 + s * nr + t);
          const double pt = __ldcg(pc + t);
          const double yv = q.dK[i] * c + (q.lam * q.dK[i] + q.rho) * pt;
          q.y[t] = yv;
          acc[0] += pt * yv;
          break;
        }
        case BP_TR_COMB: {
          double c = 0.0;
          for (int s = 0; s < q.sdf; ++s) c += __ldcg(q.cpd + s * nr + t);
          const double xt = __ldcg(q.x + t);
          const double o = __ldcg(q.bbar + t) - (q.dK[i] * c + (q.lam * q.dK[i] + q.rho) * xt);
          q.tres[t] = o;
          acc[0] += o * o;
          break;
        }
        case BP_FINAL_COMB: {
          double c = 0.0;
          for (int s = 0; s < q.sdf; ++s) c += __ldcg(q.cpd + s * nr + t);
          q.W[t] = c;
          break;
        }
        default:
          break;
      }
    }
  }
  block_sum<2>(acc, sred);
  if (threadIdx.x == 0) {
    q.red[2 * tile] = acc[0];
    q.red[2 * tile + 1] = acc[1];
  }
}

// --------------------------------------------------------- product tiles --
// Tile t = (row block t % mt, k split t / mt) of C_s = op(U_K) B over the
// split's k range, op(U_K)(i, k) = U_K[k n + i] (ATRANS: U_K itself) or
// U_K[i n + k] (U_K').  Thread (ty, tx) of the 256 owns TM = 4 rows and TN
// columns (8 TN >= r).  The next k slab is fetched into registers while the
// current one is multiplied from shared memory.

// FP32: B = fl32(D_K p) (product 1) or Yhat1 (product 2); C in cp32.  Rows
// 4 ty .. 4 ty + 3 (one 128-bit shared load per k), two smem buffers.
// Product 1 forms the new direction p = z + beta p_old (p = z after a
// restart, beta = 0) as it stages B; the tiles of the first row block store
// it (each k in exactly one of them) into the other p buffer.
template <bool ATRANS, int TN>
__device__ __noinline__ void prod32_tile(const BatchReq& q, const DevScalars& ss, int aux, int tile,
                                         float* sm) {
  constexpr int BM = kBatchBM, BK = kBK32, TM = 4, LDA = BM + 4;
  constexpr int AL = BM * BK / kThreads, BL = BK * 64 / kThreads;
  const int n = q.n, r = q.r;
  const int mt = row_blocks(q);
  const int i0 = (tile % mt) * BM, sp = tile / mt;
  const int kbeg = sp * q.kc32, kend = min(n, kbeg + q.kc32);
  const float* __restrict__ A = q.UKhi;
  const float* B = q.y132;
  const int par = (aux >> 1) & 1;
  double* pnew = q.p[par];
  const double* pold = q.p[par ^ 1];
  const double beta = ATRANS ? ss.beta : 0.0;
  const bool store_p = ATRANS && i0 == 0;
  float* As = sm;                      // [2][BK][LDA]
  float* Bs = sm + 2 * BK * LDA;       // [2][BK][64]
  const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5;
  float acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.f;
  float ra[AL], rb[BL];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + kThreads * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      const int i = i0 + ii, k = k0 + kk;
      ra[u] = (i < n && k < kend)
                  ? __ldg(ATRANS ? A + (int64_t)k * n + i : A + (int64_t)i * n + k)
                  : 0.f;
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + kThreads * u;
      const int kk = idx % BK, j = idx / BK;
      const int k = k0 + kk;
      float v = 0.f;
      if (k < kend && j < r) {
        const int64_t t = (int64_t)j * n + k;
        if (ATRANS) {
          const double zt = __ldcg(q.z + t);
          const double pv = beta != 0.0 ? zt + beta * __ldcg(pold + t) : zt;
          if (store_p) pnew[t] = pv;
          v = (float)(q.dK[k] * pv);
        } else {
          v = __ldcg(B + t);
        }
      }
      rb[u] = v;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + kThreads * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      As[(buf * BK + kk) * LDA + ii] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + kThreads * u;
      Bs[(buf * BK + idx % BK) * 64 + idx / BK] = rb[u];
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
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[(buf * BK + kk) * LDA + 4 * ty]);
      const float a[TM] = {a4.x, a4.y, a4.z, a4.w};
      float bv[TN];
#pragma unroll
      for (int c = 0; c < TN; ++c) bv[c] = Bs[(buf * BK + kk) * 64 + tx * TN + c];
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[m][c] = fmaf(a[m], bv[c], acc[m][c]);
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* C = q.cp32 + (int64_t)sp * n * r;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int i = i0 + 4 * ty + m;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int j = tx * TN + c;
      if (j < r) C[(int64_t)j * n + i] = acc[m][c];
    }
  }
}

// Double-float (FP64-accurate without the FP64 units): A = U_K as hi/lo FP32
// pairs, B an FP64 array (times D_K when `scale`) split into hi/lo as it is
// staged, exact TwoProd products and compensated sums (df.cuh); C in cpd as
// FP64.  Rows ty + 32 m of a 64-row block (the double-float accumulators
// take twice the registers of FP32 ones).
template <bool ATRANS, int TN>
__device__ __noinline__ void proddf_tile(const BatchReq& q, int tile, const double* B, bool scale,
                                         float* sm) {
  constexpr int BM = kBatchBMdf, BK = kBKdf, TM = BM / 32, LDA = BM + 1;
  constexpr int AL = BM * BK / kThreads, BL = BK * 64 / kThreads;
  const int n = q.n, r = q.r;
  const int mt = row_blocks_df(q);
  const int i0 = (tile % mt) * BM, sp = tile / mt;
  const int kbeg = sp * q.kcdf, kend = min(n, kbeg + q.kcdf);
  const float* __restrict__ Ahi = q.UKhi;
  const float* __restrict__ Alo = q.UKlo;
  float* Ash = sm;                  // [BK][LDA]
  float* Asl = Ash + BK * LDA;
  float* Bsh = Asl + BK * LDA;      // [BK][64]
  float* Bsl = Bsh + BK * 64;
  const int tid = threadIdx.x, ty = tid & 31, tx = tid >> 5;
  df acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = df{0.f, 0.f};
  float rah[AL], ral[AL], rbh[BL], rbl[BL];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + kThreads * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      const int i = i0 + ii, k = k0 + kk;
      float h = 0.f, l = 0.f;
      if (i < n && k < kend) {
        const int64_t off = ATRANS ? (int64_t)k * n + i : (int64_t)i * n + k;
        h = __ldg(Ahi + off);
        l = __ldg(Alo + off);
      }
      rah[u] = h;
      ral[u] = l;
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + kThreads * u;
      const int kk = idx % BK, j = idx / BK;
      const int k = k0 + kk;
      df d{0.f, 0.f};
      if (k < kend && j < r) {
        double v = __ldcg(B + (int64_t)j * n + k);
        if (scale) v *= q.dK[k];
        d = df_from_double(v);
      }
      rbh[u] = d.hi;
      rbl[u] = d.lo;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int u = 0; u < AL; ++u) {
      const int idx = tid + kThreads * u;
      int ii, kk;
      if (ATRANS) { ii = idx % BM; kk = idx / BM; } else { kk = idx % BK; ii = idx / BK; }
      Ash[kk * LDA + ii] = rah[u];
      Asl[kk * LDA + ii] = ral[u];
    }
#pragma unroll
    for (int u = 0; u < BL; ++u) {
      const int idx = tid + kThreads * u;
      Bsh[(idx % BK) * 64 + idx / BK] = rbh[u];
      Bsl[(idx % BK) * 64 + idx / BK] = rbl[u];
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
      df a[TM], b[TN];
#pragma unroll
      for (int m = 0; m < TM; ++m) a[m] = df{Ash[kk * LDA + ty + 32 * m], Asl[kk * LDA + ty + 32 * m]};
#pragma unroll
      for (int c = 0; c < TN; ++c) b[c] = df{Bsh[kk * 64 + tx * TN + c], Bsl[kk * 64 + tx * TN + c]};
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int c = 0; c < TN; ++c) df_acc_prod(acc[m][c], a[m], b[c]);
    }
    __syncthreads();
    if (more) stash();
    __syncthreads();
  }
  double* C = q.cpd + (int64_t)sp * n * r;
#pragma unroll
  for (int m = 0; m < TM; ++m) {
    const int i = i0 + ty + 32 * m;
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int j = tx * TN + c;
      if (j < r) C[(int64_t)j * n + i] = df_to_double(df_norm(acc[m][c]));
    }
  }
}

template <bool ATRANS>
__device__ void prod32_by_rank(const BatchReq& q, const DevScalars& ss, int aux, int tile,
                               float* sm) {
  if (q.r <= 8) prod32_tile<ATRANS, 1>(q, ss, aux, tile, sm);
  else if (q.r <= 16) prod32_tile<ATRANS, 2>(q, ss, aux, tile, sm);
  else if (q.r <= 32) prod32_tile<ATRANS, 4>(q, ss, aux, tile, sm);
  else prod32_tile<ATRANS, 8>(q, ss, aux, tile, sm);
}

template <bool ATRANS>
__device__ void proddf_by_rank(const BatchReq& q, int tile, const double* B, bool scale,
                               float* sm) {
  if (q.r <= 8) proddf_tile<ATRANS, 1>(q, tile, B, scale, sm);
  else if (q.r <= 16) proddf_tile<ATRANS, 2>(q, tile, B, scale, sm);
  else if (q.r <= 32) proddf_tile<ATRANS, 4>(q, tile, B, scale, sm);
  else proddf_tile<ATRANS, 8>(q, tile, B, scale, sm);
}

// ------------------------------------------------------ gather-dot tiles --
// Tile t = virtual warps [8 t, 8 t + 8) of the request's piece
// decomposition, one per warp of the block; Xhat rows are the sums of the
// split partials of product 1 (or of the true residual's first product).
template <int MODE, int RP, int LPO>
__device__ __noinline__ void gds_tile(const BatchReq& q, int tile, unsigned char* smem) {
  using IO = typename GdsTypes<MODE>::IO;
  using Acc = typename GdsTypes<MODE>::Acc;
  Acc* xs = reinterpret_cast<Acc*>(smem) + (threadIdx.x >> 5) * RP;
  const int w = tile * 8 + (threadIdx.x >> 5);
  if (w >= q.pl.nwarps) return;
  const bool f32 = MODE == GDS_F32;
  const IO* Xh = f32 ? reinterpret_cast<const IO*>(q.cp32) : reinterpret_cast<const IO*>(q.cpd);
  GdsXsrc src;
  src.nsum = f32 ? q.s32 : q.sdf;
  src.sum_stride = (int64_t)q.n * q.r;
  IO* Y = f32 ? reinterpret_cast<IO*>(q.y132) : reinterpret_cast<IO*>(q.y164);
  gds_warp_range<MODE, RP, LPO, false>(q.pl, w, q.zhi, nullptr, q.r, Xh, q.n, src,
                                       reinterpret_cast<IO*>(q.gds_partial), Y, q.n, nullptr,
                                       nullptr, nullptr, xs);
}

__device__ void gds32_by_rank(const BatchReq& q, int tile, unsigned char* smem) {
  if (q.r <= 8) gds_tile<GDS_F32, 8, 1>(q, tile, smem);
  else if (q.r <= 16) gds_tile<GDS_F32, 16, 1>(q, tile, smem);
  else if (q.r <= 32) gds_tile<GDS_F32, 32, 1>(q, tile, smem);
  else if (q.r <= 40) gds_tile<GDS_F32, 40, 1>(q, tile, smem);
  else if (q.r <= 48) gds_tile<GDS_F32, 48, 1>(q, tile, smem);
  else gds_tile<GDS_F32, 64, 2>(q, tile, smem);
}

__device__ void gdsdf_by_rank(const BatchReq& q, int tile, unsigned char* smem) {
  if (q.r <= 8) gds_tile<GDS_DF, 8, 1>(q, tile, smem);
  else if (q.r <= 16) gds_tile<GDS_DF, 16, 1>(q, tile, smem);
  else if (q.r <= 32) gds_tile<GDS_DF, 32, 2>(q, tile, smem);
  else if (q.r <= 48) gds_tile<GDS_DF, 48, 4>(q, tile, smem);
  else gds_tile<GDS_DF, 64, 4>(q, tile, smem);
}

// ------------------------------------------------------------- finalizer --
// Run by the whole block that finished the last tile of phase `ph` of a
// request: adds the tiles' partial sums in tile order (deterministic), then
// thread 0 takes the PCG's decisions on the request's scalars and opens the
// next phase.  The decisions mirror the step-by-step solve: alpha = (r, z) /
// (p, A p); beta = (r, z)_new / (r, z); the recurrence reaching tol or
// max_iter ends the cycle early; every k iterations (or at such an end) the
// FP64-accurate true residual decides convergence, and a restart from it
// when the cycle ended or the recurrence drifted below a quarter of it.
// Returns the next phase in thread 0 (other threads: BP_DONE).
__device__ __noinline__ int decide(BatchLocal& L, BatchState* S, int ph, int ntiles,
                                   double* sred) {
  const BatchReq& q = L.q;
  const bool sums = ph == BP_RHS_COMB || ph == BP_RESTART || ph == BP_COMB2 ||
                    ph == BP_UPDATE || ph == BP_TR_COMB;
  double tot[2] = {0.0, 0.0};
  if (sums) {
    for (int t = threadIdx.x; t < ntiles; t += kThreads) {
      tot[0] += __ldcg(q.red + 2 * t);
      tot[1] += __ldcg(q.red + 2 * t + 1);
    }
    block_sum<2>(tot, sred);
  }
  if (threadIdx.x != 0) return BP_DONE;
  DevScalars* s = &L.s;
  BatchLocal* vs = &L;
  int next = BP_DONE;
  switch (ph) {
    case BP_SETUP:
      if (*(volatile const int*)q.err != 0) {
        *(volatile int*)&S->fail = 1;
        next = BP_DONE;
      } else {
        next = BP_RHS_PROD;
      }
      break;
    case BP_RHS_PROD:
      next = BP_RHS_COMB;
      break;
    case BP_RHS_COMB:
      s->bb = tot[0];
      if (tot[0] == 0.0) {  // b = 0: W = 0 solves the system exactly
        s->done = 1;
        next = BP_FINAL_PROD;
      } else {
        vs->adopt = 0;
        next = BP_RESTART;
      }
      break;
    case BP_RESTART:
      s->rr = tot[1];
      s->beta = 0.0;
      s->restarts = s->restarts + 1;
      s->rz = tot[0];
      vs->adopt = 0;
      vs->chunk = 0;
      if (!isfinite(tot[0])) {
        s->status = CPHIFI_E_BREAKDOWN;
        s->done = 1;
        next = BP_FINAL_PROD;
      } else {
        next = BP_PROD1;
      }
      break;
    case BP_PROD1:
      next = BP_GDS;
      break;
    case BP_GDS:
      next = BP_PROD2;
      break;
    case BP_PROD2:
      next = BP_COMB2;
      break;
    case BP_COMB2: {
      s->pAp = tot[0];
      const double a = s->rz / tot[0];
      if (!(tot[0] > 0.0) || !isfinite(a)) {
        s->status = CPHIFI_E_BREAKDOWN;
        s->done = 1;
        next = BP_FINAL_PROD;
      } else {
        s->alpha = a;
        next = BP_UPDATE;
      }
      break;
    }
    case BP_UPDATE: {
      const double rz_new = tot[0];
      s->rr = tot[1];
      s->iter = s->iter + 1;
      const double beta = rz_new / s->rz;
      s->beta = beta;
      if (!isfinite(beta) || !isfinite(tot[1])) {
        s->status = CPHIFI_E_BREAKDOWN;
        s->done = 1;
      }
      if (tot[1] <= q.tol2 * s->bb) s->inner_done = 1;
      if (s->iter >= q.max_iter) s->inner_done = 1;
      s->rz = rz_new;
      vs->iters = s->iter;
      vs->chunk = vs->chunk + 1;
      next = s->done ? BP_FINAL_PROD
                     : (s->inner_done || vs->chunk >= q.k_replace ? BP_TR_PROD1 : BP_PROD1);
      break;
    }
    case BP_TR_PROD1:
      next = BP_TR_GDS;
      break;
    case BP_TR_GDS:
      next = BP_TR_PROD2;
      break;
    case BP_TR_PROD2:
      next = BP_TR_COMB;
      break;
    case BP_TR_COMB: {
      const double trr = tot[0];
      s->true_rr = trr;
      s->true_evals = s->true_evals + 1;
      if (!isfinite(trr)) {
        s->status = CPHIFI_E_BREAKDOWN;
        s->done = 1;
        next = BP_FINAL_PROD;
        break;
      }
      s->done = (trr <= q.tol2 * s->bb) ? 1 : 0;
      if (s->done) {
        next = BP_FINAL_PROD;
      } else if (s->inner_done || s->rr < 0.25 * trr) {
        if (q.max_iter - s->iter <= 0) {
          next = BP_FINAL_PROD;  // max_iter: the last true residual stands
        } else {
          s->rr = trr;  // the true residual replaces the recurrence residual
          s->inner_done = 0;
          vs->adopt = 1;
          next = BP_RESTART;
        }
      } else {
        vs->chunk = 0;
        next = BP_PROD1;
      }
      break;
    }
    case BP_FINAL_PROD:
      next = BP_FINAL_COMB;
      break;
    default:
      next = BP_DONE;
      break;
  }
  if (next == BP_PROD1) vs->par = vs->par ^ 1;  // the new direction goes to the other buffer
  // write the decisions back (no wait: the fence before the next phase is
  // published orders them)
  volatile DevScalars* gs = q.s;
  gs->rz = s->rz;
  gs->pAp = s->pAp;
  gs->alpha = s->alpha;
  gs->beta = s->beta;
  gs->rr = s->rr;
  gs->bb = s->bb;
  gs->true_rr = s->true_rr;
  gs->iter = s->iter;
  gs->inner_done = s->inner_done;
  gs->done = s->done;
  gs->status = s->status;
  gs->true_evals = s->true_evals;
  gs->restarts = s->restarts;
  volatile BatchState* gst = S;
  gst->chunk = vs->chunk;
  gst->adopt = vs->adopt;
  gst->par = vs->par;
  gst->iters = vs->iters;
  gst->phase = next;
  return next;
}

// Thread 0: publishes the next phase of a request (its claim word with no
// tile claimed), or its completion.
// With `take`, the caller keeps the first tile of the new phase (the claim
// word is published with one tile claimed).
__device__ void open_phase(const BatchLocal& L, BatchState* S, BatchCtl* ctl, int next,
                           bool take) {
  *(volatile unsigned*)&S->done = 0u;
  __threadfence();
  const int nt = phase_tiles(L.q, next);
  atomicExch(&S->claim, claim_word(nt, next, L.adopt | (L.par << 1)) + (take && nt > 0 ? 1 : 0));
  if (next == BP_DONE) {
    *(volatile long long*)&S->t_done = global_ns();
    __threadfence();
    atomicAdd(&ctl->completed, 1u);
  }
}

// ---------------------------------------------------------------- kernel --
__device__ void run_tile(const BatchLocal& L, int ph, int aux, int tile, unsigned char* smem,
                         double* sred) {
  const BatchReq& q = L.q;
  float* smf = reinterpret_cast<float*>(smem);
  switch (ph) {
    case BP_RHS_PROD: proddf_by_rank<false>(q, tile, q.Bm, false, smf); break;
    case BP_PROD1: prod32_by_rank<true>(q, L.s, aux, tile, smf); break;
    case BP_GDS: gds32_by_rank(q, tile, smem); break;
    case BP_PROD2: prod32_by_rank<false>(q, L.s, aux, tile, smf); break;
    case BP_TR_PROD1: proddf_by_rank<true>(q, tile, q.x, true, smf); break;
    case BP_TR_GDS: gdsdf_by_rank(q, tile, smem); break;
    case BP_TR_PROD2: proddf_by_rank<false>(q, tile, q.y164, false, smf); break;
    case BP_FINAL_PROD: proddf_by_rank<true>(q, tile, q.x, false, smf); break;
    default: vec_tile(ph, q, L.s, aux, tile, smem, sred); break;
  }
}

// The block's copy of request jr: the descriptor (unless already held), the
// scalars and the state, in one round of independent loads.
__device__ __forceinline__ void load_local(const BatchReq* __restrict__ reqs, const BatchState* st,
                                           const DevScalars* scal, int jr, bool have_q,
                                           BatchLocal& L) {
  constexpr int kQW = sizeof(BatchReq) / 4, kSW = sizeof(DevScalars) / 8;
  static_assert(sizeof(BatchReq) % 4 == 0 && sizeof(DevScalars) % 8 == 0, "word copies");
  static_assert(kQW <= 128 && kSW <= 32, "one load per thread");
  const int t = threadIdx.x;
  if (!have_q && t < kQW)
    reinterpret_cast<unsigned*>(&L.q)[t] = __ldg(reinterpret_cast<const unsigned*>(reqs + jr) + t);
  if (t >= 128 && t < 128 + kSW)
    reinterpret_cast<unsigned long long*>(&L.s)[t - 128] =
        __ldcg(reinterpret_cast<const unsigned long long*>(scal + jr) + (t - 128));
  if (t == 160) L.chunk = __ldcg(&st[jr].chunk);
  if (t == 161) L.adopt = __ldcg(&st[jr].adopt);
  if (t == 162) L.par = __ldcg(&st[jr].par);
  if (t == 163) L.iters = __ldcg(&st[jr].iters);
}

__global__ void __launch_bounds__(kThreads, 2)
batch_kernel(const BatchReq* __restrict__ reqs, BatchState* st, const DevScalars* scal,
             BatchCtl* ctl, int nreq, long long timeout_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sred[64];
  __shared__ int s_min[kThreads / 32];
  __shared__ int s_req, s_tile, s_ntiles, s_phase, s_aux, s_exit, s_fin, s_held;
  __shared__ __align__(16) BatchLocal L;
  unsigned seen = 0xffffffffu;
  long long t_last = global_ns();
  unsigned backoff = 32;
  if (threadIdx.x == 0) {
    s_held = -1;
    atomicCAS(reinterpret_cast<unsigned long long*>(&ctl->t_start), 0ull,
              (unsigned long long)t_last);
  }
  for (;;) {
    // the request with an unclaimed tile that has run the most iterations
    // (a long chain so far is likely to stay long), the first in the given
    // order among equals: key = iterations << 16 | (65535 - index)
    unsigned key = 0;
    for (int j = threadIdx.x; j < nreq; j += kThreads) {
      const unsigned long long w = *(volatile unsigned long long*)&st[j].claim;
      const int it = *(volatile int*)&st[j].iters;
      if ((int)claim_count(w) < claim_tiles(w))
        key = max(key, ((unsigned)min(it, 32767) << 16) | (unsigned)(65535 - j));
    }
    key = __reduce_max_sync(0xffffffffu, key);
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = (int)key;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned kb = 0;
      for (int k = 0; k < kThreads / 32; ++k) kb = max(kb, (unsigned)s_min[k]);
      const int c = kb ? 65535 - (int)(kb & 0xffffu) : INT_MAX;
      s_req = -1;
      s_exit = 0;
      if (c != INT_MAX) {
        const unsigned long long old = atomicAdd(&st[c].claim, 1ull);
        if ((int)claim_count(old) < claim_tiles(old)) {
          __threadfence();
          s_req = c;
          s_tile = (int)claim_count(old);
          s_ntiles = claim_tiles(old);
          s_phase = claim_phase(old);
          s_aux = claim_aux(old);
        }
      }
      if (s_req < 0) {
        if (*(volatile unsigned*)&ctl->completed >= (unsigned)nreq ||
            *(volatile int*)&ctl->abort)
          s_exit = 1;
      }
    }
    __syncthreads();
    if (s_exit) break;
    const int jr = s_req;
    if (jr < 0) {
      // nothing to claim: wait, bounded by the progress of the whole launch
      if (threadIdx.x == 0) {
        const unsigned pr = *(volatile unsigned*)&ctl->progress;
        const long long now = global_ns();
        if (pr != seen) {
          seen = pr;
          t_last = now;
        } else if (now - t_last > timeout_ns) {
          ctl->err = 1;
          atomicExch(&ctl->abort, 1);
        }
        __nanosleep(backoff);
        backoff = min(backoff * 2u, kSleepMaxNs);
      }
      __syncthreads();
      continue;
    }
    backoff = 32;
    load_local(reqs, st, scal, jr, s_held == jr, L);
    __syncthreads();
    if (threadIdx.x == 0) s_held = jr;
    // this tile, and while this block closes phases, the first tile of each
    // next phase (the request's chain goes on without waiting for a poll)
    for (;;) {
      run_tile(L, s_phase, s_aux, s_tile, smem, sred);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->progress, 1u);
        const unsigned d = atomicAdd(&st[jr].done, 1u);
        s_fin = d == (unsigned)s_ntiles - 1u;
        if (s_fin) __threadfence();
      }
      __syncthreads();
      if (!s_fin) break;
      const int nx = decide(L, &st[jr], s_phase, s_ntiles, sred);
      if (threadIdx.x == 0) {
        const int nt = phase_tiles(L.q, nx);
        open_phase(L, &st[jr], ctl, nx, true);
        s_fin = nx != BP_DONE && nt > 0;
        s_tile = 0;
        s_ntiles = nt;
        s_phase = nx;
        s_aux = L.adopt | (L.par << 1);
      }
      __syncthreads();
      if (!s_fin) break;
    }
  }
}

// Dynamic shared memory: the largest tile layout (FP32 product: two slabs
// of A and B; double-float product: hi/lo slabs; restart/update: U_V and two
// 32-row buffers; gather: 8 warps x 64 double-float entries).
constexpr size_t kSmemProd32 = (2 * kBK32 * (kBatchBM + 4) + 2 * kBK32 * 64) * sizeof(float);
constexpr size_t kSmemProdDf = (2 * kBKdf * (kBatchBMdf + 1) + 2 * kBKdf * 64) * sizeof(float);
constexpr size_t kSmemPrecond = (kMaxRank * kMaxRank + 2 * kBatchRows * (kMaxRank + 1)) * sizeof(float);
constexpr size_t kSmemGds = 8 * kMaxRank * sizeof(df);
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kBatchSmem = cmax(cmax(kSmemProd32, kSmemProdDf), cmax(kSmemPrecond, kSmemGds));

}  // namespace

unsigned long long batch_first_claim(const BatchReq& q) {
  return claim_word(phase_tiles(q, BP_SETUP), BP_SETUP, 0);
}

int batch_blocks(int num_sms) {
  int occ = 0;
  if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kBatchSmem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, kThreads, kBatchSmem) !=
      cudaSuccess)
    return 0;
  return occ < 1 ? 0 : occ * num_sms;
}

cudaError_t launch_batch(const BatchReq* reqs, BatchState* st, const DevScalars* scal,
                         BatchCtl* ctl, int nreq, long long timeout_ns, int blocks,
                         cudaStream_t stream) {
  if (nreq <= 0) return cudaSuccess;
  if (blocks < 1) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBatchSmem);
  if (e != cudaSuccess) return e;
  batch_kernel<<<blocks, kThreads, kBatchSmem, stream>>>(reqs, st, scal, ctl, nreq, timeout_ns);
  return cudaGetLastError();
}

}  // namespace cphifi
