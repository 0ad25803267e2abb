// Host-side launchers of the solver's kernels (one declaration per kernel
// family; definitions live beside the kernels).  All take a stream and
// return the cudaError_t of the launch.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace cphifi {

// ---------------------------------------------------------------- obs.cu ---
// Kernel indices in [0, n) (else bit 1 of *err) and, with `sorted`,
// non-decreasing (else bit 4).  The Zhat build checks the other modes'
// indices (bit 1) and the values' finiteness (bit 2).
cudaError_t launch_validate_kidx(const int32_t* kidx, int64_t q, int n, bool sorted, int* err,
                                 cudaStream_t st);
cudaError_t launch_validate_dense(const double* a, int64_t count, int* err,
                                  cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs by key < 2^key_bits.
// tmp must hold radix_sort_tmp_bytes(q) bytes.  On return keys/vals hold the
// sorted sequence.
size_t radix_sort_tmp_bytes(int64_t q);
cudaError_t radix_sort_pairs(uint32_t* keys, int32_t* vals, int64_t q,
                             int key_bits, void* tmp, cudaStream_t st);
cudaError_t launch_iota(int32_t* v, int64_t q, cudaStream_t st);
cudaError_t launch_row_ptr(const uint32_t* sorted_keys, int64_t q, int n,
                           int64_t* row_ptr, cudaStream_t st);
// Pieces: the kernel-index segments cut at multiples of L (each warp of the
// gather-dot/scatter owns L sorted observations); every index owns >= 1 piece.
// A non-null `gate` that reads nonzero (an input error found by an earlier
// kernel) makes these kernels, and the Zhat build, return without touching
// memory: their inputs cannot be trusted to stay in range.
cudaError_t launch_piece_counts(const int64_t* row_ptr, int n, int64_t L,
                                int32_t* seg_count, const int* gate, cudaStream_t st);
cudaError_t launch_piece_fill(const int64_t* row_ptr, int n, int64_t L,
                              const int32_t* seg_first, const int32_t* seg_count,
                              int32_t* pseg, int32_t* pbeg, int32_t* pend,
                              const int* gate, cudaStream_t st);
cudaError_t launch_warp_first(const int32_t* pbeg, int npieces, const int32_t* np_dev,
                              int64_t L, int W, int32_t* warp_first, const int* gate,
                              cudaStream_t st);
// Exclusive scan of int32 counts into int32 offsets (out has n+1 entries).
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n,
                               void* tmp, size_t tmp_bytes, cudaStream_t st);
size_t exclusive_scan_tmp_bytes(int64_t n);
// Zhat storage: tiles of 32 sorted observations, each a 32 x r column-major
// block; (l, j) lives at zidx(l, j, ts) with tile stride ts.  The FP64 copy
// has ts = 32 r; the FP32 pair is one array whose tiles hold the hi block
// then the lo block (ts = 64 r, lo = hi + 32 r), so a pass over the hi parts
// alone keeps touching the same pages as one over both.  A buffer holds
// zhat_elems(q, r) values per part.
__host__ __device__ __forceinline__ int64_t zidx(int64_t l, int j, int64_t ts) {
  return (l >> 5) * ts + 32 * (int64_t)j + (l & 31);
}
__host__ __device__ __forceinline__ int64_t zhat_elems(int64_t q, int r) {
  return ((q + 31) >> 5) * 32 * (int64_t)r;
}
// Conversions between the FP64 copy and the interleaved FP32 pair.
cudaError_t launch_zhat_split(const double* z64, int64_t q, int r, float* zhl, cudaStream_t st);
cudaError_t launch_zhat_join(const float* zhl, int64_t q, int r, double* z64, cudaStream_t st);
// Gather-dot/scatter (Eqs. vl and yhat1) over the piece decomposition.
struct PieceList {
  const int32_t* seg;
  const int32_t* beg;
  const int32_t* end;
  const int32_t* seg_first;
  const int32_t* seg_count;
  unsigned* seg_ticket;
  const int32_t* warp_first;  // nwarps + 1
  int npieces;
  int nwarps;
  // Optional dynamic assignment (2 counters, zero between launches): physical
  // warps draw the ranges (and the Zhat build its tile chunks) from wctr[0],
  // so blocks that start late -- their SM held by another stream's kernel --
  // take less work instead of running their fixed share after all others.
  // The last warp to finish resets both counters.  NULL: static shares.
  unsigned* wctr = nullptr;
};
// Gather-dot/scatter in three arithmetics (all in the tiled Zhat layout):
// FP32 reading Zhat's hi part (mixed operator), FP64 reading z64 (FP64
// operator), double-float reading hi + lo (FP64-accurate true residuals).
cudaError_t launch_gds_f32(const PieceList& pl, const float* zhi, int r, const float* Xh,
                           int64_t xld, float* partial, float* Y, int64_t yld,
                           const DevScalars* skip, cudaStream_t st);
cudaError_t launch_gds_f64(const PieceList& pl, const double* z64, int r, const double* Xh,
                           int64_t xld, double* partial, double* Y, int64_t yld,
                           const DevScalars* skip, cudaStream_t st);
cudaError_t launch_gds_df(const PieceList& pl, const float* zhi, const float* zlo, int r,
                          const double* Xh, int64_t xld, double* partial, double* Y,
                          int64_t yld, const DevScalars* skip, cudaStream_t st);
// Zhat (Eq. zhat) in sorted order, computed in double-float from the
// factors' interleaved hi/lo rows (fhl[m], see launch_split_rows_df) and
// written as hi/lo FP32 pairs (zhi, tiles [hi | lo]) and/or FP64 (z64), and
// in the same pass the MTTKRP B(i,:) = sum_{i_l = i} t_l Zhat(l,:) (B
// column-major, ld ldb, FP64-accurate), over the pieces of pl (its own
// decomposition; pl.wctr required).  perm = NULL: input already sorted.  B is
// written for every kernel index (zero rows for empty ones); bad other-mode
// indices set *err bit 1, non-finite values bit 2.  partial: pl.npieces x 64
// doubles.  [w_begin, w_end) restricts a launch to those virtual warps (-1:
// all), so that the pass can follow a chunked upload of the observations.
cudaError_t launch_zhat_mttkrp_fused(const PieceList& pl, int64_t q, const int32_t* perm,
                                     const int32_t* oidx, int d_other, const float* const* fhl,
                                     const int64_t* sizes_dev, int r, const double* vals,
                                     float* zhi, double* z64, double* partial, double* B,
                                     int64_t ldb, int* err, const int* gate, int num_sms,
                                     cudaStream_t st, int w_begin = 0, int w_end = -1);

// -------------------------------------------------------------- dense.cu ---
// Skinny product C = op(A) diag(s) B for A n x n (op = identity when a_trans
// is true, transpose otherwise, see dense.cu), B n x ncols column-major; the
// k-range is split over `nsplit` blocks of columns of A and the partial
// products land in C + split * split_stride.
template <typename TA, typename TC>
cudaError_t launch_gemm_skinny(const TA* A, int64_t lda, bool a_trans,
                               const double* scale_k, const TC* B, int64_t ldb,
                               TC* C, int64_t ldc, int64_t split_stride,
                               int n, int ncols, int nsplit,
                               const DevScalars* skip, cudaStream_t st);
template <typename TA, typename TC>
int gemm_pick_split(int n, int num_sms);
// Double-float product C = op(A) B with A = Ahi + Alo and B = Bhi + Blo
// (hi/lo FP32 pairs), FP64 partial products per split.
cudaError_t launch_gemm_df(const float* Ahi, const float* Alo, int64_t lda, bool a_trans,
                           const float* Bhi, const float* Blo, int64_t ldb, double* C,
                           int64_t ldc, int64_t split_stride, int n, int ncols, int nsplit,
                           const DevScalars* skip, cudaStream_t st);
int gemm_df_pick_split(int n, int num_sms);
// Row-major interleaved hi/lo split of a column-major rows x cols matrix X:
// hl[2 (i*cols + j)] + hl[2 (i*cols + j) + 1] = X[i + rows*j] (a 32-byte sector
// holds 4 consecutive elements of a row, hi and lo together).
cudaError_t launch_split_rows_df(const double* X, int64_t rows, int cols, float* hl,
                                 cudaStream_t st);
// hi + lo = scale[t % rows] * X[t] (scale may be NULL), t < total.
cudaError_t launch_split_df(const double* X, const double* scale, int64_t rows, int64_t total,
                            float* hi, float* lo, cudaStream_t st);

// ------------------------------------------------------------ tc_gemm.cu ---
// tcgen05 products C_split = A B (TF32 or BF16 operands, FP32 accumulation);
// A and B are K-major and described by TMA tensor maps (tc_make_map).
bool tc_available(int n);
cudaError_t tc_make_map(CUtensorMap* map, const void* base, bool bf16, uint64_t inner,
                        uint64_t outer, uint64_t row_stride_bytes, uint32_t box_outer);
int tc_pad_cols(int ncols);
int tc_pick_split(int n, int num_sms);
// mal/mbl (TF32 only, may be NULL): maps of the lo parts of a 3-term split
// product A_hi B_hi + A_hi B_lo + A_lo B_hi.
cudaError_t launch_tc_gemm(bool bf16, const CUtensorMap& ma, const CUtensorMap& mb,
                           const CUtensorMap* mal, const CUtensorMap* mbl, float* C, int64_t ldc,
                           int64_t split_stride, int n, int ncols, int nsplit,
                           const DevScalars* skip, int* err, cudaStream_t st);
// ------------------------------------------------------------ oz_gemm.cu ---
// FP64-accurate products op(U_K) B on the tensor cores from 7 BF16 slices of
// each operand (error-free splitting, exact group sums in TMEM).  U_K slices:
// a1 (rows of U_K), a2 (rows of U_K'), BF16 [7][oz_mpad(n)][ldt] each, with
// the row exponents e[0..n) (a1) and e[n..2n) (a2).  B slices: BF16
// [7][64][ldt] (r <= 64 rows used, the rest zero) with column exponents
// cexp[0..r).  C_split gets
// FP64 partial products over nsplit ranges of k (oz_pick_split).  slices = 3
// uses the first 3 slices of each operand only (the products of slice index
// sum <= 2): per term a few 2^-24 of the row and column scales, the
// low-precision operator of CPHIFI_MIXED_BF16X3.
int64_t oz_mpad(int n);
size_t oz_uk_bytes(int n, int64_t ldt);
size_t oz_b_bytes(int r, int64_t ldt);
cudaError_t launch_oz_uk(const double* U, int n, int64_t ldt, __nv_bfloat16* a1, __nv_bfloat16* a2,
                         int* e, cudaStream_t st);
cudaError_t oz_make_maps(const __nv_bfloat16* a1, const __nv_bfloat16* a2, int n, int64_t ldt,
                         CUtensorMap* m1, CUtensorMap* m2);
cudaError_t oz_make_b_map(const __nv_bfloat16* b, int n, int r, int64_t ldt, CUtensorMap* m);
// B'(k, j) = scale[k] B(k, j) (scale may be NULL), B column-major with ld ldb.
cudaError_t launch_oz_b(const double* B, const double* scale, int n, int r, int64_t ldb,
                        int64_t ldt, __nv_bfloat16* out, int* cexp, const DevScalars* skip,
                        cudaStream_t st);
int oz_pick_split(int n, int num_sms);
cudaError_t launch_oz_gemm(const CUtensorMap& ma, const int* rexp, const CUtensorMap& mb,
                           const int* cexp, double* C, int64_t ldc, int64_t split_stride, int n,
                           int ncols, int nsplit, const DevScalars* skip, int* err,
                           cudaStream_t st, int slices = 7);

// TF32 hi/lo split (hi = x with 13 low bits cleared, lo = x - hi).
cudaError_t launch_tf32_split(const float* src, float* hi, float* lo, int64_t total,
                              cudaStream_t st);
cudaError_t launch_tf32_split_block(const float* x, int64_t ldx, int64_t rows, int64_t total,
                                    float* hi, float* lo, int64_t ldo, const DevScalars* skip,
                                    cudaStream_t st);
// U_K -> T copy with leading dimension ldo, transposed (row-major U_K) or not.
template <typename T>
cudaError_t launch_uk_copy(const double* U, int n, int64_t ldo, bool transpose, T* out,
                           cudaStream_t st);
// out(i, j) = T(scale[i] X(i, j)) at j*ldo + i for an n x r column-major X
// (ld n; scale may be NULL).
template <typename TS, typename T>
cudaError_t launch_scale_to(const TS* X, const double* scale, int64_t rows, int64_t total, T* out,
                            int64_t ldo, cudaStream_t st);

// ----------------------------------------------------------------- cg.cu ---
cudaError_t launch_gram(const double* const* factors_dev, const int64_t* sizes_host,
                        int d_other, int r, double* V, cudaStream_t st);
cudaError_t launch_jacobi_eig(const double* V, int r, double* dV, double* UV,
                              int max_sweeps, int* info, cudaStream_t st);
cudaError_t launch_build_D(const double* dK, const double* dV, int n, int r,
                           double gamma, double lam, double rho, double* D64,
                           float* D32, cudaStream_t st);

enum CombineMode {
  CM_STORE = 0,  // out = sum_s C_s
  CM_DK = 1,     // out = dK .* sum_s C_s
  CM_APPLY = 2,  // out = dK .* sum_s C_s + (lam dK + rho) .* V; pAp -> alpha
  CM_RESID = 3,  // out = Bv - (dK .* sum_s C_s + (lam dK + rho) .* V); ||out||^2 -> true residual
  CM_DK_NORM = 4, // out = dK .* sum_s C_s; ||out||^2 -> bb (the right-hand side)
  CM_TRUE = 5     // as CM_RESID into a separate buffer: sets true_rr and the
                  // convergence flag, leaves the recurrence (rr, inner_done) alone
};
// res = tres, rr = true_rr, inner_done = 0: the true residual of CM_TRUE
// replaces the recurrence residual (before a restart).
cudaError_t launch_adopt_residual(const double* tres, double* res, int64_t count, DevScalars* s,
                                  cudaStream_t st);
// C (nsplit partials of n x r, split_stride apart) is consumed: its contents
// are undefined afterwards (the lines are dropped from L2 without write-back).
template <typename TC, typename TO>
cudaError_t launch_combine(int mode, const TC* C, int64_t split_stride, int nsplit,
                           int n, int r, const double* dK, const double* V,
                           const double* Bv, TO* out, DevScalars* s,
                           RedScratch red, const DevScalars* skip, cudaStream_t st);

enum UpdateMode {
  UP_ITER = 0,     // x += a p; r -= a y; z = M^-1 r; (r,z), ||r||^2 -> beta
  UP_RESTART = 1   // z = M^-1 r; (r,z) -> rz, beta = 0
};
template <typename TP>
cudaError_t launch_update_precond(int mode, int n, int r, double* x, double* rres,
                                  const double* p, const double* y, double* z,
                                  const TP* UV, const TP* D, DevScalars* s,
                                  RedScratch red, cudaStream_t st);
// p = z + beta p; and the operand of the next n x n product, in type TB:
// pop(i, j) = TB(scale[i] p(i, j)) at j*ldp + i (scale may be NULL), plus a
// BF16 copy when pop16 is set.
template <typename TB>
cudaError_t launch_pupdate(int n, int r, const double* z, double* p, TB* pop,
                           const double* scale, int64_t ldp, __nv_bfloat16* pop16,
                           DevScalars* s, cudaStream_t st);
cudaError_t launch_precond_only(int n, int r, const double* X, double* Y,
                                const double* UV, const double* D, cudaStream_t st);
template <typename TS, typename TD>
cudaError_t launch_convert(const TS* src, TD* dst, int64_t count, cudaStream_t st);

// --------------------------------------------------------------- gram.cu ---
// Per-index Gram blocks C_i = sum_{i_l = i} Zhat(l,:)'Zhat(l,:) (n blocks of
// r x r, row-major, symmetric) over the pieces of pl (a decomposition of the
// sorted observations; the exact piece count at np_dev, the capacity in
// pl.npieces; partial: capacity x r^2 values): FP32 from Zhat's hi parts, or
// FP64-accurate (double-float) from the hi/lo pair zhi or, when zhi is NULL,
// the FP64 copy z64.  And Yhat1(i,:) = C_i Xhat(i,:)' for all i.
cudaError_t launch_gram_build_f32(const PieceList& pl, const int32_t* np_dev, int grid,
                                  const float* zhi, int r, float* partial, float* C,
                                  cudaStream_t st);
cudaError_t launch_gram_build_df(const PieceList& pl, const int32_t* np_dev, int grid,
                                 const float* zhi, const double* z64, int r, double* partial,
                                 double* C, cudaStream_t st);
cudaError_t launch_gram_apply_f32(const float* C, int n, int r, const float* Xh, int64_t xld,
                                  float* Y, int64_t yld, const DevScalars* skip,
                                  cudaStream_t st);
cudaError_t launch_gram_apply_f64(const double* C, int n, int r, const double* Xh, int64_t xld,
                                  double* Y, int64_t yld, const DevScalars* skip,
                                  cudaStream_t st);

// ------------------------------------------------------------ kpoints.cu ---
// K(i, j) = k(x_i, x_j) from n points (row-major n x dim) for the Gaussian or
// Matern-3/2 kernel (cphifi_kernel_kind) with the given bandwidth: the whole
// K (FP64), or Y = K X (X, Y n x r column-major) with K's tiles generated on
// the fly in FP64 or FP32.
cudaError_t launch_kpoints_build(const double* pts, int n, int dim, int kind, double bandwidth,
                                 double* K, cudaStream_t st);
// nsplit > 1: the column range of K split over nsplit blocks per row block,
// their partial products in `part` (nsplit x n x r doubles), added in split
// order into Y.  kpoints_pick_split: the split that fills the GPU.
int kpoints_pick_split(int n, int num_sms);
cudaError_t launch_kpoints_apply(bool fp64, const double* pts, int n, int dim, int kind,
                                 double bandwidth, int r, const double* X, double* Y,
                                 int nsplit, double* part, cudaStream_t st);

// ---------------------------------------------------------------- eig.cu ---
// FP64 symmetric eigendecomposition by parallel two-sided Jacobi (Eq. eigK):
// A (n x n, column-major; the lower triangle is read) is overwritten by the
// eigenvectors in the order of the eigenvalues w (ascending).  Synchronous on
// st; returns a cphifi_status, with the reason in *why on failure.
constexpr int kSymEigMaxN = 4096;
constexpr int kSymEigMaxSweeps = 60;
int sym_eig_jacobi(double* A, int n, double* w, cudaStream_t st, std::string* why);
int sym_eig_max_n();

// ---------------------------------------------------------------- als.cu ---
// The alternating fit (§2).  keep_obs: kidx_s = sorted keys, and the
// other-mode indices / values of observation perm[l] (l without perm) in the
// sorted order.  mode_keys: keys[l] = oidx_s[l d_other + m].  als_rows: the
// CP-ALS update of finite mode m (r x r normal equations per row of A_m,
// FP64, Cholesky; Ak = K W, n x r; factors/sizes: device arrays of the
// d_other factor pointers (column-major n_m x r) and sizes; writes Anew, may
// alias factors[m]; *nfail counts rows with observations kept unchanged).
// fit: out[0] = sum (t - m)^2, out[1] = sum t^2 of the model.
cudaError_t launch_keep_obs(int64_t q, int d_other, const uint32_t* keys, const int32_t* perm,
                            const int32_t* oidx, const double* vals, int32_t* kidx_s,
                            int32_t* oidx_s, double* vals_s, const int* gate, cudaStream_t st);
cudaError_t launch_mode_keys(int64_t q, int d_other, int m, const int32_t* oidx_s, uint32_t* keys,
                             cudaStream_t st);
cudaError_t launch_als_rows(int n_m, int m, int d_other, int r, int n, const int64_t* row_ptr_m,
                            const int32_t* perm_m, const int32_t* kidx_s, const int32_t* oidx_s,
                            const double* vals_s, const double* Ak, const double* const* factors,
                            const int64_t* sizes, double* Anew, int* nfail, int num_sms,
                            cudaStream_t st);
cudaError_t launch_fit(int64_t q, int d_other, int r, int n, const int32_t* kidx_s,
                       const int32_t* oidx_s, const double* vals_s, const double* Ak,
                       const double* const* factors, const int64_t* sizes, RedScratch red,
                       double* out, int num_sms, cudaStream_t st);

// -------------------------------------------------------------- batch.cu ---
// Many mixed-FP32 PCG solves in one persistent launch.  Each request is a
// chain of phases (set-up, right-hand side, restart, the six phases of an
// iteration, the four of the FP64-accurate true residual, the final
// W = U_K x); a phase is a set of independent tiles.  Blocks claim tiles
// from the requests' claim words (requests in the order given, the first
// with an unclaimed tile first); the block that finishes the last tile of a
// phase reduces the phase's partial sums in tile order, takes the decisions
// of the PCG (step sizes, convergence, restart) and opens the next phase.
// No tile ever waits for another, so blocks need not be co-resident; an idle
// block polls, and every block leaves when all requests are done, or when no
// tile finished anywhere for `timeout_ns` (error 1 in BatchCtl::err).
constexpr int kBatchRows = 32;    // rows of a vector tile
constexpr int kBatchBM = 128;     // rows of an FP32 product tile
constexpr int kBatchBMdf = 64;    // rows of a double-float product tile
constexpr int kBatchPhaseDone = 15;  // BatchState::phase of a finished request
struct BatchReq {
  int n = 0, r = 0;
  int s32 = 1, sdf = 1;           // k-range splits of the FP32 / double-float products
  int kc32 = 0, kcdf = 0;         // their k chunks
  int max_iter = 0, k_replace = 10;
  double tol2 = 0.0, lam = 0.0, rho = 0.0, gamma = 0.0;
  const float* UKhi = nullptr;    // U_K = UKhi + UKlo (n x n column-major)
  const float* UKlo = nullptr;
  const double* dK = nullptr;     // eigenvalues of K
  const double* dV = nullptr;     // eigenvalues of V
  const float* UV32 = nullptr;    // eigenvectors of V (r x r)
  PieceList pl{};                 // gather-dot/scatter decomposition (static shares)
  const float* zhi = nullptr;     // Zhat hi/lo tiles
  const double* Bm = nullptr;     // sparse MTTKRP B (n x r)
  const int* err = nullptr;       // input error word of the problem's creation
  double *x = nullptr, *res = nullptr, *z = nullptr, *y = nullptr, *bbar = nullptr,
         *tres = nullptr, *D64 = nullptr, *y164 = nullptr;
  double* p[2] = {nullptr, nullptr};  // the direction, alternating between two buffers
  float *D32 = nullptr, *y132 = nullptr;
  float* cp32 = nullptr;          // s32 x n x r split partials
  double* cpd = nullptr;          // sdf x n x r split partials
  void* gds_partial = nullptr;    // npieces x 64 values
  double* red = nullptr;          // 2 per vector tile
  DevScalars* s = nullptr;
  double* W = nullptr;            // n x r result (column-major)
};
struct alignas(64) BatchState {
  unsigned long long claim = 0;   // open phase, its tiles, tiles claimed (batch.cu)
  unsigned done = 0;              // tiles of the open phase finished
  int phase = 0;
  int chunk = 0;                  // iterations since the last true residual
  int adopt = 0;                  // the next restart starts from the true residual
  int par = 0;                    // p[par] is the current direction
  int iters = 0;                  // PCG iterations so far (the claim priority)
  int fail = 0;                   // input error found at set-up
  long long t_done = 0;           // global timer (ns) when the request finished
};
struct BatchCtl {
  unsigned completed = 0;         // requests finished
  unsigned progress = 0;          // tiles finished, all requests
  int abort = 0;
  int err = 0;                    // 1: no tile finished within timeout_ns
  long long t_start = 0;          // global timer (ns) when the first block started
};
// First claim word of a request (its set-up phase).
unsigned long long batch_first_claim(const BatchReq& q);
// Blocks of the persistent launch on this device, and the launch itself.
int batch_blocks(int num_sms);
cudaError_t launch_batch(const BatchReq* reqs, BatchState* st, const DevScalars* scal,
                         BatchCtl* ctl, int nreq, long long timeout_ns, int blocks,
                         cudaStream_t stream);  // scal: reqs[j].s == scal + j

}  // namespace cphifi
