// The gather-dot/scatter of the matrix-free product (Eqs. vl and yhat1,
// §4.4.1) for one virtual warp of the piece decomposition, shared by the
// stand-alone kernel (obs.cu) and the persistent batch kernel (batch.cu).
//
// Warp w owns the pieces [warp_first[w], warp_first[w+1]), i.e. the sorted
// observations [w L, (w+1) L).  Per piece (one kernel index i), each
// observation l is handled by LPO lanes (each owning RP/LPO of the columns):
// they load Zhat(l, :) (a warp round reads one contiguous tile), form
// xbar_l = Xhat(i,:).Zhat(l,:) (Eq. vl; partial dots summed across the LPO
// lanes) and accumulate xbar_l Zhat(l,:) in registers (Eq. yhat1).  The warp
// then sums its partial rows; a kernel index covered by one piece is written
// directly, otherwise each piece stores its row and the last piece to finish
// (per-index ticket) adds the pieces in piece order.  No floating-point
// atomics: the result is deterministic.
//
// Arithmetic modes:
//   GDS_F32 : FP32 throughout, Zhat = hi        (the mixed-precision operator)
//   GDS_F64 : FP64 throughout, Zhat = z64        (the FP64 operator)
//   GDS_DF  : double-float (df.cuh), Zhat = hi + lo, Xhat and Yhat1 FP64
//             (FP64-accurate true residuals of the mixed solve)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "launch.h"

namespace cphifi {

// Cross-lane helpers for LPO lanes per observation: lane = sub * OPW + o with
// OPW = 32 / LPO observations per warp round; the lane owns the CPL = RP/LPO
// columns [sub*CPL, (sub+1)*CPL).
template <typename T, int LPO>
__device__ __forceinline__ T sum_over_subs(T v) {
  constexpr int OPW = 32 / LPO;
#pragma unroll
  for (int o = OPW; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums acc over the OPW observations of a sub-group and stores the row piece:
// lane (sub, o) writes columns sub*CPL + c for c = o, o + OPW, ...
template <typename T, int RP, int LPO>
__device__ __forceinline__ void reduce_row(T (&acc)[RP / LPO]) {
  constexpr int OPW = 32 / LPO, CPL = RP / LPO;
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int o = OPW >> 1; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
}

// Writes a reduced row (columns < r) to Y(:, seg) or, when the kernel index is
// split over several pieces, to the piece's partial row; the last piece to
// finish sums the partial rows in piece order.
template <typename T, int RP, int LPO>
__device__ __forceinline__ void store_row(const PieceList& pl, int p, int seg, int r,
                                          const T (&acc)[RP / LPO], T* __restrict__ partial,
                                          T* __restrict__ Y, int64_t yld) {
  constexpr int OPW = 32 / LPO, CPL = RP / LPO;
  const int lane = threadIdx.x & 31, sub = lane / OPW, o = lane % OPW;
  const int np = pl.seg_count[seg];
  if (np == 1) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int j = sub * CPL + c;
      if ((c % OPW) == o && j < r) Y[(int64_t)j * yld + seg] = acc[c];
    }
    return;
  }
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int j = sub * CPL + c;
    if ((c % OPW) == o && j < r) partial[(int64_t)p * RP + j] = acc[c];
  }
  __threadfence();
  __syncwarp();
  unsigned t = 0;
  if (lane == 0) t = atomicAdd(&pl.seg_ticket[seg], 1u);
  t = __shfl_sync(0xffffffffu, t, 0);
  if (t == (unsigned)(np - 1)) {
    __threadfence();
    const int f = pl.seg_first[seg];
    for (int j = lane; j < r; j += 32) {
      T sacc = T(0);
      for (int k = 0; k < np; ++k) sacc += __ldcg(&partial[(int64_t)(f + k) * RP + j]);
      Y[(int64_t)j * yld + seg] = sacc;
    }
    if (lane == 0) pl.seg_ticket[seg] = 0u;
  }
}

enum { GDS_F32 = 0, GDS_F64 = 1, GDS_DF = 2 };

template <int MODE>
struct GdsTypes;
template <>
struct GdsTypes<GDS_F32> { using IO = float; using Acc = float; };
template <>
struct GdsTypes<GDS_F64> { using IO = double; using Acc = double; };
template <>
struct GdsTypes<GDS_DF> { using IO = double; using Acc = df; };

__device__ __forceinline__ void acc_fma(float& a, float x, float y) { a = fmaf(x, y, a); }
__device__ __forceinline__ void acc_fma(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void acc_fma(df& a, df x, df y) { df_acc_prod(a, x, y); }
__device__ __forceinline__ float acc_zero(float) { return 0.f; }
__device__ __forceinline__ double acc_zero(double) { return 0.0; }
__device__ __forceinline__ df acc_zero(df) { return df{0.f, 0.f}; }
__device__ __forceinline__ float acc_out(float a) { return a; }
__device__ __forceinline__ double acc_out(double a) { return a; }
__device__ __forceinline__ double acc_out(df a) { return df_to_double(df_norm(a)); }

// Where the row Xhat(i, :) comes from.  Stand-alone (nsum = 0): Xh(i, j) at
// Xh[j xld + i], read through the read-only path.  Batch kernel (nsum >= 1):
// the row is the sum, in split order, of nsum partial products at
// Xh + s sum_stride, read through L2 (it was written by other blocks of the
// same launch), summed in FP64 and rounded once to the IO type.
struct GdsXsrc {
  int nsum = 0;
  int64_t sum_stride = 0;
};

// WTS (weights mode): xbar_l is a given weight t_l (wts[wperm[l]], or wts[l]
// without a permutation) instead of the dot product, so Y(i,:) =
// sum_{i_l = i} t_l Zhat(l,:), a sparse MTTKRP over a stored Zhat.
// xs: this warp's RP-entry row buffer in shared memory.
template <int MODE, int RP, int LPO, bool WTS>
__device__ __forceinline__ void gds_warp_range(
    const PieceList& pl, int w, const float* __restrict__ zhi, const double* __restrict__ z64,
    int r, const typename GdsTypes<MODE>::IO* __restrict__ Xh, int64_t xld, GdsXsrc xsrc,
    typename GdsTypes<MODE>::IO* __restrict__ partial, typename GdsTypes<MODE>::IO* __restrict__ Y,
    int64_t yld, const double* __restrict__ wts, const int32_t* __restrict__ wperm,
    const float2* __restrict__ wdf, typename GdsTypes<MODE>::Acc* xs) {
  using IO = typename GdsTypes<MODE>::IO;
  using Acc = typename GdsTypes<MODE>::Acc;
  constexpr int OPW = 32 / LPO, CPL = RP / LPO;
  const int lane = threadIdx.x & 31, sub = lane / OPW, o = lane % OPW;
  const int p_end = pl.warp_first[w + 1];
  for (int p = pl.warp_first[w]; p < p_end; ++p) {
    const int seg = pl.seg[p];
    const int b = pl.beg[p], e = pl.end[p];
    if (b == e) {  // an index without observations (its own single piece): a zero row
      for (int j = lane; j < r; j += 32) Y[(int64_t)j * yld + seg] = IO(0);
      continue;
    }
    if constexpr (!WTS) {
      __syncwarp();
      for (int j = lane; j < RP; j += 32) {
        IO v = IO(0);
        if (j < r) {
          if (xsrc.nsum == 0) {
            v = Xh[(int64_t)j * xld + seg];
          } else {
            double t = 0.0;
            for (int s = 0; s < xsrc.nsum; ++s)
              t += (double)__ldcg(Xh + s * xsrc.sum_stride + (int64_t)j * xld + seg);
            v = (IO)t;
          }
        }
        if constexpr (MODE == GDS_DF) xs[j] = df_from_double(v);
        else xs[j] = v;
      }
      __syncwarp();
    }
    Acc acc[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) acc[c] = acc_zero(Acc());
    // Zhat values of the OPW observations of the round starting at l0
    auto load = [&](int l0, Acc (&z)[CPL]) {
      const int l = l0 + o;
      const bool act = l < e;
      // hi/lo pair: tile stride 64 r (lo block at +32 r); FP64: 32 r
      const int64_t base = zidx(act ? l : b, 0, (MODE == GDS_F64 ? 32 : 64) * (int64_t)r);
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = sub * CPL + c;
        const bool ld = act && j < r;
        if constexpr (MODE == GDS_F32) z[c] = ld ? __ldcs(zhi + base + 32 * j) : 0.f;
        else if constexpr (MODE == GDS_F64) z[c] = ld ? __ldcs(z64 + base + 32 * j) : 0.0;
        else z[c] = ld ? df{__ldcs(zhi + base + 32 * j), __ldcs(zhi + base + 32 * (r + j))}
                       : df{0.f, 0.f};
      }
    };
    // double-float with 4 lanes per observation (r > 32): the next round's
    // values are loaded while this round's arithmetic (half of the pass's
    // time) runs; with fewer lanes the extra registers would spill
    constexpr bool kPrefetch = MODE == GDS_DF && LPO >= 4;
    Acc zn[kPrefetch ? CPL : 1];
    if constexpr (kPrefetch) load(b, zn);
    // Every lane runs the same number of rounds so the cross-lane sums of
    // the dot product see the whole warp.
    for (int l0 = b; l0 < e; l0 += OPW) {
      const int l = l0 + o;
      const bool act = l < e;
      Acc z[CPL];
      if constexpr (kPrefetch) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) z[c] = zn[c];
        if (l0 + OPW < e) load(l0 + OPW, zn);
      } else {
        load(l0, z);
      }
      Acc xb;
      if constexpr (WTS) {
        if constexpr (MODE == GDS_DF) {
          const float2 t2 = act ? __ldcs(wdf + l) : make_float2(0.f, 0.f);
          xb = df{t2.x, t2.y};
        } else {
          const double t = act ? wts[wperm ? (int64_t)wperm[l] : (int64_t)l] : 0.0;
          xb = (Acc)t;
        }
      } else {
        Acc dot = acc_zero(Acc());
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc_fma(dot, xs[sub * CPL + c], z[c]);
        if constexpr (MODE == GDS_DF) {
          df d = df_norm(dot);
          // sum the partial dots of the LPO lanes of this observation
#pragma unroll
          for (int s = OPW; s < 32; s <<= 1) {
            const df other{__shfl_xor_sync(0xffffffffu, d.hi, s),
                           __shfl_xor_sync(0xffffffffu, d.lo, s)};
            d = df_add(d, other);
          }
          xb = d;
        } else {
          xb = LPO > 1 ? sum_over_subs<Acc, LPO>(dot) : dot;
        }
      }
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc_fma(acc[c], xb, z[c]);
    }
    IO accd[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) accd[c] = (IO)acc_out(acc[c]);
    reduce_row<IO, RP, LPO>(accd);
    store_row<IO, RP, LPO>(pl, p, seg, r, accd, partial, Y, yld);
  }
}

}  // namespace cphifi
