// FP64-accurate skinny products on the tensor cores by error-free operand
// splitting (the splitting scheme of Ozaki, Ogita, Oishi and Rump, 2012):
// C = op(U_K) B for the FP64-accurate steps of the mixed solve (the
// right-hand side D_K U_K' B, the true residual's U_K (D_K x̄) and U_K' Ŷ1,
// and W = U_K x̄; Eq. unaligned-infinite-1 in the eigenbasis of §4.4).
//
// Splitting.  Every row i of A (the output row) is scaled by 2^-e_i so that
// its largest entry is below 1, every column j of B by 2^-f_j likewise, and
// each scaled value v is cut into S = 7 slices
//     v = sum_t m_t 2^(-7-8t) + rest,   |m_t| <= 128 integer,  |rest| <= 2^-56,
// by rounding the remainder to the grid of the slice (m_t = rint(rest 2^(7+8t))).
// Each slice has at most 8 significant bits, so it is exact in BF16, and
// the product of two slices, m_t m_u 2^(-14-8(t+u)), is exact in FP32.
//
// Products.  C_ij 2^-(e_i+f_j) = sum_{t+u <= 6} (A_t B_u)_ij up to 2^-53 of
// the row/column scales.  The slice products are grouped by g = t + u: all
// terms of a group are integer multiples of the group's unit 2^(-14-8g) and
// bounded by 2^14 units, so a group's sum over a 256-wide k chunk, at most
// (g+1) 256 2^14 <= 2^24 units for g <= 3, is exact in an FP32 accumulator
// whatever the order of the additions.  Each group has its own TMEM
// accumulator; those of groups 0..3 (10 products) are read after every chunk
// and added into double-float registers, those of groups 4..6 (18 products,
// at most 2^-32 of the result) accumulate over the whole k range, their FP32
// rounding far below the result's last bit.  The result is FP64-accurate
// (about 2^-50 of sum_k |A_ik B_kj|, like the double-float product it
// replaces) at tensor-core speed.
//
// Layout.  A slices: BF16 [7][mpad][ldt], slice t's row i at row t mpad + i
// of one K-major tensor map (mpad = n rounded up to 128).  B slices: BF16
// [7][64][ldt], slice u's column j at row 64 u + j (rows r..63 zero).  Row
// and column exponents e_i, f_j as int arrays.
//
// Block: 10 warps.  Warp 8 (one lane) streams 128-byte k slabs with TMA: per
// slab the 7 B slices (one ring slot, each slice padded to 64 rows) and the 7
// A slices (one ring stage each); warp 9 (one lane) issues the products: for
// A_t, the slices B_0..B_{6-t} are contiguous in shared memory, so one
// tcgen05.mma with N = 64 m covers m <= 4 of them and writes group t + u to
// the TMEM region of that group (64 columns each, 7 regions): 10 MMAs per
// 16 k instead of 28.  Warps 0..7 drain every chunk: warp w reads TMEM lanes
// 32 (w % 4).. and columns (w / 4) NP/2.. of the regions 0..3, one output row
// per thread, and adds them into double-float registers (the MMA issuer
// overwrites them in the next chunk once they are read); the regions 4..6
// are read once at the end.  Every wait is bounded (error code, then TMEM is
// freed and the kernel returns).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "launch.h"
#include "tc_util.cuh"

namespace cphifi {

using namespace tcu;

namespace {

constexpr int kOzS = 7;               // slices per operand
constexpr int kOzBRows = 64;          // rows of one B slice (r padded with zero rows)
constexpr int kOzChunkSlabs = 4;      // 4 slabs of 64 k = 256 k per exact chunk
constexpr int kOzDrainWarps = 8;
constexpr int kOzThreads = (kOzDrainWarps + 2) * 32;
constexpr int kOzABytes = 128 * 128;  // one A slice tile: 128 rows x 128 bytes
constexpr int kOzAStages = 6;
constexpr int kOzBBytes = kOzS * kOzBRows * 128;  // the 7 B slices of one slab
constexpr size_t kOzSmem = (size_t)kOzAStages * kOzABytes + 2 * kOzBBytes + 1024;
constexpr uint32_t kOzTmemCols = 512;  // 7 group regions of 64 columns

// Eight consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

// Reads the group regions [G0, G1) (NH columns each, this thread's half),
// releases them to the MMA issuer through `bar` when `release`, then adds
// them into acc.
template <int NH, int G0, int G1>
__device__ __forceinline__ void oz_drain(uint32_t tbase, df (&acc)[NH], uint64_t* bar,
                                         bool release) {
  uint32_t v[G1 - G0][NH];
#pragma unroll
  for (int g = G0; g < G1; ++g)
#pragma unroll
    for (int c0 = 0; c0 < NH; c0 += 8)
      tmem_ld8(tbase + 64u * g + c0, *reinterpret_cast<uint32_t(*)[8]>(&v[g - G0][c0]));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  if (release) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(bar);
  }
#pragma unroll
  for (int g = 0; g < G1 - G0; ++g)
#pragma unroll
    for (int c = 0; c < NH; ++c) df_acc_add(acc[c], df{__uint_as_float(v[g][c]), 0.f});
}

}  // namespace

// S: slices of each operand that take part (7: FP64-accurate; 3: products
// t + u <= 2 of 8-bit slices, FP32-level accuracy: per term the truncated
// slices, 2^-24 (|a| + |b|), and the dropped products of index sum 3 and 4,
// at most 2 2^-24 + 2^-32, of the row and column scales; for the
// low-precision operator).  The layouts are those of the 7 slices; only the
// first S of each operand are loaded.
template <int NP, int S>
__global__ void __launch_bounds__(kOzThreads, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               int mpad, const int* __restrict__ rexp, const int* __restrict__ cexp,
               double* __restrict__ C, int64_t ldc, int64_t split_stride, int n, int ncols,
               int kchunk, const DevScalars* skip, int* err) {
  if (dev_skip(skip)) return;
  static_assert(S >= 1 && S <= kOzS, "slice count");
  constexpr int NH = NP / 2;  // columns per drain thread
  constexpr int GX = S < 4 ? S : 4;  // groups read after every chunk (exact sums)
  extern __shared__ uint8_t smem_raw[];
  // ex_lo: the drain has read the group regions 0..3 of a chunk
  __shared__ uint64_t a_full[kOzAStages], a_empty[kOzAStages], b_full[2], b_empty[2], ex_full,
      ex_lo;
  __shared__ uint32_t tmem_slot;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* bring = smem + kOzAStages * kOzABytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  const int kbeg = blockIdx.y * kchunk;
  const int kend = min(n, kbeg + kchunk);
  const int nslab = kend > kbeg ? (kend - kbeg + 63) / 64 : 0;
  const int nch = (nslab + kOzChunkSlabs - 1) / kOzChunkSlabs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzAStages; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    mbar_init(&ex_full, 1);
    mbar_init(&ex_lo, kOzDrainWarps * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kOzTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == kOzDrainWarps) {
    if (lane == 0) {  // producer: B slices per slab (2-slot ring), A slices one stage each
      bool ok = true;
      for (int c = 0; c < nslab && ok; ++c) {
        const int k0 = kbeg + c * 64;
        const int bs = c & 1;
        if (c >= 2 && !mbar_wait(&b_empty[bs], (uint32_t)((c >> 1) & 1) ^ 1u, err, 1)) break;
        mbar_expect_tx(&b_full[bs], S * kOzBRows * 128);
        for (int u = 0; u < S; ++u)
          tma_load_2d(bring + bs * kOzBBytes + u * kOzBRows * 128, &tmB, k0, u * kOzBRows,
                      &b_full[bs]);
        for (int t = 0; t < S; ++t) {
          const int idx = c * S + t, s = idx % kOzAStages;
          if (idx >= kOzAStages &&
              !mbar_wait(&a_empty[s], (uint32_t)((idx / kOzAStages) & 1) ^ 1u, err, 1)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&a_full[s], kOzABytes);
          tma_load_2d(smem + s * kOzABytes, &tmA, k0, t * mpad + m0, &a_full[s]);
        }
      }
    }
  } else if (warp == kOzDrainWarps + 1) {
    if (lane == 0) {  // MMA issuer
      // descriptors of stage 0 / slot 0; other stages, slices and k offsets
      // add (byte offset >> 4) to the start-address field
      const uint64_t da0 = sdesc(smem), db0 = sdesc(bring);
      bool ok = true;
      for (int c = 0; c < nslab && ok; ++c) {
        const int ch = c / kOzChunkSlabs;
        const bool first = (c % kOzChunkSlabs) == 0;
        if (first && ch > 0)  // the previous chunk's exact group sums were read
          ok = mbar_wait(&ex_lo, (uint32_t)((ch - 1) & 1), err, 8);
        const int bs = c & 1;
        if (!ok || !mbar_wait(&b_full[bs], (uint32_t)((c >> 1) & 1), err, 2)) break;
        const uint64_t dbs = db0 + (uint64_t)((bs * kOzBBytes) >> 4);
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const int idx = c * S + t, s = idx % kOzAStages;
          if (!mbar_wait(&a_full[s], (uint32_t)((idx / kOzAStages) & 1), err, 2)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t das = da0 + (uint64_t)((s * kOzABytes) >> 4);
          // B_u0 .. B_{u0+m-1} in one MMA of N = 64 m into regions t+u0 ..
#pragma unroll
          for (int u0 = 0; u0 < S - t; u0 += 4) {
            const int m = min(4, S - t - u0);
            const uint32_t id = idesc<__nv_bfloat16>(64 * m);
            const uint32_t d = tmem + 64u * (uint32_t)(t + u0);
            const uint64_t db = dbs + (uint64_t)((u0 * kOzBRows * 128) >> 4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // the chunk's first products overwrite regions 0..3 (exact
              // per chunk); regions 4..6 accumulate over the whole k range
              const bool fresh = t == 0 && kk == 0 && (u0 == 0 ? first : c == 0);
              mma<__nv_bfloat16>(d, das + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), id,
                                 fresh ? 0u : 1u);
            }
          }
          mma_commit(&a_empty[s]);
        }
        if (!ok) break;
        mma_commit(&b_empty[bs]);
        if ((c % kOzChunkSlabs) == kOzChunkSlabs - 1 || c == nslab - 1) mma_commit(&ex_full);
      }
    }
  } else {
    // drain: the exact group sums of every chunk (regions 0..3), then the
    // rest (regions 4..6, accumulated over the k range), into double-float
    // registers
    const int quad = warp & 3, half = warp >> 2;
    const int row = m0 + quad * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * NH);
    df acc[NH];
#pragma unroll
    for (int c = 0; c < NH; ++c) acc[c] = df{0.f, 0.f};
    bool ok = true;
    for (int ch = 0; ch < nch; ++ch) {
      ok = ok && mbar_wait(&ex_full, (uint32_t)(ch & 1), err, 4);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if constexpr (NH <= 24 || GX <= 2) {
        oz_drain<NH, 0, GX>(tbase, acc, &ex_lo, true);
      } else {  // fewer registers in flight
        oz_drain<NH, 0, 2>(tbase, acc, &ex_lo, false);
        oz_drain<NH, 2, GX>(tbase, acc, &ex_lo, true);
      }
    }
    if constexpr (S > 4) {
      if (nch > 0) oz_drain<NH, 4, S>(tbase, acc, &ex_lo, false);
    }
    if (row < n && (ok || nslab == 0)) {
      const int ei = rexp[row];
      double* Cs = C + (int64_t)blockIdx.y * split_stride;
#pragma unroll
      for (int c = 0; c < NH; ++c) {
        const int j = half * NH + c;
        if (j < ncols) {
          const df a = df_norm(acc[c]);
          Cs[(int64_t)j * ldc + row] = ldexp((double)a.hi + (double)a.lo, ei + cexp[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOzTmemCols)
                 : "memory");
}

// ------------------------------------------------------------ splitting ---

// Scaled slices of one value v in (-1, 1) (already scaled by its row or
// column exponent), in 64-bit fixed point: M = v 2^62, then for t = 0..6
// m_t = round(M / 2^(55-8t)) (ties up), M -= m_t 2^(55-8t); slice t =
// m_t 2^(-7-8t) with |m_t| <= 128, and |v - sum_t slice_t| <= 2^-56.
// Non-finite input: every slice NaN (the product then reports it).
__device__ __forceinline__ void oz_slices(double v, __nv_bfloat16 (&s)[kOzS]) {
  if (!isfinite(v)) {
#pragma unroll
    for (int t = 0; t < kOzS; ++t) s[t] = __float2bfloat16_rn(__int_as_float(0x7fc00000));
    return;
  }
  long long M = __double2ll_rn(ldexp(v, 62));
#pragma unroll
  for (int t = 0; t < kOzS; ++t) {
    const int sh = 55 - 8 * t;
    const long long m = (M + (1LL << (sh - 1))) >> sh;
    M -= m * (1LL << sh);
    s[t] = __float2bfloat16_rn(ldexpf((float)m, sh - 62));  // exact: |m| <= 128
  }
}

// Exponent e with max|.| < 2^e (0 for a zero or non-finite maximum).
__device__ __forceinline__ int oz_exponent(double mx) {
  if (!(mx > 0.0) || !isfinite(mx)) return 0;
  int e;
  frexp(mx, &e);
  return e;
}

// Exponents of the row maxima of U_K (column-major n x n): e[i], i < n, for
// the rows of U_K (A of U_K X), one thread per row (reads coalesced across
// the threads); e[n + j] for its columns (the rows of U_K', A of U_K' X), one
// warp per column.
__global__ void oz_uk_row_exponents_kernel(const double* __restrict__ U, int n, int* e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double mx = 0.0;
  bool fin = true;
  for (int k = 0; k < n; ++k) {
    const double v = U[(int64_t)k * n + i];
    fin = fin && isfinite(v);
    mx = fmax(mx, fabs(v));
  }
  e[i] = fin ? oz_exponent(mx) : 0;
}

__global__ void oz_uk_col_exponents_kernel(const double* __restrict__ U, int n, int* e) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= n) return;
  double mx = 0.0;
  bool fin = true;
  for (int k = lane; k < n; k += 32) {
    const double v = U[(int64_t)j * n + k];
    fin = fin && isfinite(v);
    mx = fmax(mx, fabs(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  fin = __all_sync(0xffffffffu, fin);
  if (lane == 0) e[n + j] = fin ? oz_exponent(mx) : 0;
}

// Slices of U_K in one orientation: transpose (A1, row-major U_K: out row i,
// element k = U(i, k)) or not (A2, row-major U_K': out row j, element k =
// U(k, j)); 32 x 32 tiles staged in shared memory so that reads and writes
// are both coalesced.  Slice t of row i is at out[(t mpad + i) ldt + k].
__global__ void oz_uk_slices_kernel(const double* __restrict__ U, int n, bool transpose,
                                    const int* __restrict__ rexp, int64_t mpad, int64_t ldt,
                                    __nv_bfloat16* __restrict__ out) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int i = bx + threadIdx.x, j = by + k;
    tile[k][threadIdx.x] = (i < n && j < n) ? U[(int64_t)j * n + i] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    int orow, ocol;
    double v;
    if (transpose) {
      orow = bx + k;
      ocol = by + threadIdx.x;
      v = tile[threadIdx.x][k];
    } else {
      orow = by + k;
      ocol = bx + threadIdx.x;
      v = tile[k][threadIdx.x];
    }
    if (orow < n && ocol < n) {
      __nv_bfloat16 s[kOzS];
      oz_slices(ldexp(v, -rexp[orow]), s);
#pragma unroll
      for (int t = 0; t < kOzS; ++t) out[((int64_t)t * mpad + orow) * ldt + ocol] = s[t];
    }
  }
}

// B operand of one product: B'(k, j) = scale[k] B(k, j) (scale may be NULL).
// Column exponents first: each block reduces the frexp exponents of 1024
// entries of one column and raises cexp[j] (preset to kOzExpNone) with one
// atomicMax; a non-finite entry raises it to kOzExpBad.
constexpr int kOzExpNone = (int)0x80808080;  // the byte pattern of the preset
constexpr int kOzExpBad = 1 << 20;

__global__ void oz_b_exponents_kernel(const double* __restrict__ B,
                                      const double* __restrict__ scale, int n, int64_t ldb,
                                      int* __restrict__ cexp, const DevScalars* skip) {
  if (dev_skip(skip)) return;
  __shared__ int red[8];
  const int j = blockIdx.y;
  int e = kOzExpNone;
  for (int u = 0; u < 4; ++u) {
    const int k = blockIdx.x * 1024 + u * 256 + threadIdx.x;
    if (k < n) {
      const double v = scale ? scale[k] * B[(int64_t)j * ldb + k] : B[(int64_t)j * ldb + k];
      if (!isfinite(v)) {
        e = kOzExpBad;
      } else if (v != 0.0) {
        int ev;
        frexp(v, &ev);
        e = max(e, ev);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    if (m != kOzExpNone) atomicMax(&cexp[j], m);
  }
}

// Slices of B' (one thread per entry); slice u of column j at
// out[(u 64 + j) ldt + k].  An all-zero column keeps exponent 0 (zero
// slices); a non-finite one gets NaN slices.
__global__ void oz_b_slices_kernel(const double* __restrict__ B, const double* __restrict__ scale,
                                   int n, int64_t ldb, int64_t ldt,
                                   __nv_bfloat16* __restrict__ out, const int* __restrict__ cexp,
                                   const DevScalars* skip) {
  if (dev_skip(skip)) return;
  const int j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int f = cexp[j];
  double v = scale ? scale[k] * B[(int64_t)j * ldb + k] : B[(int64_t)j * ldb + k];
  if (f >= kOzExpBad) v = __longlong_as_double(0x7ff8000000000000LL);
  __nv_bfloat16 sl[kOzS];
  oz_slices(f == kOzExpNone || f >= kOzExpBad ? v : ldexp(v, -f), sl);
#pragma unroll
  for (int u = 0; u < kOzS; ++u) out[((int64_t)u * kOzBRows + j) * ldt + k] = sl[u];
}

// The product's exponent of column j (0 for an all-zero column).
__global__ void oz_b_fix_exponents_kernel(int* cexp, int r, const DevScalars* skip) {
  if (dev_skip(skip)) return;
  const int j = threadIdx.x;
  if (j < r && (cexp[j] == kOzExpNone || cexp[j] >= kOzExpBad)) cexp[j] = 0;
}

// ------------------------------------------------------------------ host ---

int64_t oz_mpad(int n) { return ((int64_t)n + 127) / 128 * 128; }

size_t oz_uk_bytes(int n, int64_t ldt) {
  return 2 * (size_t)kOzS * oz_mpad(n) * ldt * sizeof(__nv_bfloat16) + 2 * (size_t)n * sizeof(int);
}

size_t oz_b_bytes(int r, int64_t ldt) {
  (void)r;
  return (size_t)kOzS * kOzBRows * ldt * sizeof(__nv_bfloat16) + 64 * sizeof(int);
}

cudaError_t launch_oz_uk(const double* U, int n, int64_t ldt, __nv_bfloat16* a1, __nv_bfloat16* a2,
                         int* e, cudaStream_t st) {
  const int64_t mpad = oz_mpad(n);
  const size_t slice_bytes = (size_t)kOzS * mpad * ldt * sizeof(__nv_bfloat16);
  cudaError_t err;
  if ((err = cudaMemsetAsync(a1, 0, slice_bytes, st)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(a2, 0, slice_bytes, st)) != cudaSuccess) return err;
  oz_uk_row_exponents_kernel<<<(n + 255) / 256, 256, 0, st>>>(U, n, e);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  oz_uk_col_exponents_kernel<<<(int)(((int64_t)n * 32 + 255) / 256), 256, 0, st>>>(U, n, e);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
  oz_uk_slices_kernel<<<grid, block, 0, st>>>(U, n, true, e, mpad, ldt, a1);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  oz_uk_slices_kernel<<<grid, block, 0, st>>>(U, n, false, e + n, mpad, ldt, a2);
  return cudaGetLastError();
}

cudaError_t oz_make_maps(const __nv_bfloat16* a1, const __nv_bfloat16* a2, int n, int64_t ldt,
                         CUtensorMap* m1, CUtensorMap* m2) {
  const uint64_t rows = (uint64_t)kOzS * oz_mpad(n);
  cudaError_t e = tc_make_map(m1, a1, true, n, rows, ldt * 2, 128);
  if (e != cudaSuccess) return e;
  return tc_make_map(m2, a2, true, n, rows, ldt * 2, 128);
}

cudaError_t oz_make_b_map(const __nv_bfloat16* b, int n, int r, int64_t ldt, CUtensorMap* m) {
  (void)r;
  return tc_make_map(m, b, true, n, (uint64_t)kOzS * kOzBRows, ldt * 2, (uint32_t)kOzBRows);
}

cudaError_t launch_oz_b(const double* B, const double* scale, int n, int r, int64_t ldb,
                        int64_t ldt, __nv_bfloat16* out, int* cexp, const DevScalars* skip,
                        cudaStream_t st) {
  if (r < 1 || r > 64) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(cexp, 0x80, (size_t)r * sizeof(int), st);
  if (e != cudaSuccess) return e;
  oz_b_exponents_kernel<<<dim3((n + 1023) / 1024, r), 256, 0, st>>>(B, scale, n, ldb, cexp, skip);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  oz_b_slices_kernel<<<dim3((n + 255) / 256, r), 256, 0, st>>>(B, scale, n, ldb, ldt, out, cexp,
                                                               skip);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  oz_b_fix_exponents_kernel<<<1, 64, 0, st>>>(cexp, r, skip);
  return cudaGetLastError();
}

int oz_pick_split(int n, int num_sms) {
  const int mt = (n + 127) / 128;
  int s = num_sms / mt;  // one wave of one block per SM (the block holds ~215 KB)
  const int chunks = (n + 255) / 256;
  if (s > chunks) s = chunks;
  if (s > 64) s = 64;
  return s < 1 ? 1 : s;
}

template <int NP, int S>
static cudaError_t oz_launch(const CUtensorMap& ma, int mpad, const int* rexp, const CUtensorMap& mb,
                             const int* cexp, double* C, int64_t ldc, int64_t split_stride, int n,
                             int ncols, int nsplit, const DevScalars* skip, int* err,
                             cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<NP, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int kchunk = (n + nsplit - 1) / nsplit;
  kchunk = (kchunk + 255) / 256 * 256;  // whole exact chunks per split
  const dim3 grid((n + 127) / 128, nsplit);
  oz_gemm_kernel<NP, S><<<grid, kOzThreads, kOzSmem, st>>>(ma, mb, mpad, rexp, cexp, C, ldc,
                                                           split_stride, n, ncols, kchunk, skip,
                                                           err);
  return cudaGetLastError();
}

template <int S>
static cudaError_t oz_by_cols(const CUtensorMap& ma, int mpad, const int* rexp,
                              const CUtensorMap& mb, const int* cexp, double* C, int64_t ldc,
                              int64_t split_stride, int n, int ncols, int nsplit,
                              const DevScalars* skip, int* err, cudaStream_t st) {
  switch (tc_pad_cols(ncols)) {
    case 16: return oz_launch<16, S>(ma, mpad, rexp, mb, cexp, C, ldc, split_stride, n, ncols, nsplit, skip, err, st);
    case 32: return oz_launch<32, S>(ma, mpad, rexp, mb, cexp, C, ldc, split_stride, n, ncols, nsplit, skip, err, st);
    case 48: return oz_launch<48, S>(ma, mpad, rexp, mb, cexp, C, ldc, split_stride, n, ncols, nsplit, skip, err, st);
    default: return oz_launch<64, S>(ma, mpad, rexp, mb, cexp, C, ldc, split_stride, n, ncols, nsplit, skip, err, st);
  }
}

cudaError_t launch_oz_gemm(const CUtensorMap& ma, const int* rexp, const CUtensorMap& mb,
                           const int* cexp, double* C, int64_t ldc, int64_t split_stride, int n,
                           int ncols, int nsplit, const DevScalars* skip, int* err,
                           cudaStream_t st, int slices) {
  const int mpad = (int)oz_mpad(n);
  if (slices == 3)
    return oz_by_cols<3>(ma, mpad, rexp, mb, cexp, C, ldc, split_stride, n, ncols, nsplit, skip,
                         err, st);
  if (slices != kOzS) return cudaErrorInvalidValue;
  return oz_by_cols<kOzS>(ma, mpad, rexp, mb, cexp, C, ldc, split_stride, n, ncols, nsplit, skip,
                          err, st);
}

}  // namespace cphifi
