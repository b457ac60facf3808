// Internal declarations shared by the CUDA translation units of libtrals.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/trals.h"

namespace trk {

// Bits of the device-side error record (one uint32 per context).
enum : unsigned {
  kErrSingular = 1u,    // non-positive pivot or zero core
  kErrBadIndex = 2u,    // a caller-provided sample index out of range
  kErrTimeout = 4u,     // a bounded device wait expired
};

constexpr int kMaxModes = TR_MAX_MODES;
constexpr int kMaxL = TR_MAX_RANK_PRODUCT;

// ------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
//   (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by the Weyl increments (W0, W1) between rounds.
// ------------------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// 53-bit uniform in [0, 1) from a (hi, lo) word pair.
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  const uint64_t bits = ((static_cast<uint64_t>(hi) << 32) | lo) >> 11;
  return static_cast<double>(bits) * 0x1.0p-53;
}

// ------------------------------------------------------------------------------------
// Launchers (defined in the .cu files; all asynchronous on `st`).
// ------------------------------------------------------------------------------------
struct SampleArgs {
  const double* p[kMaxModes];    // per ring position m
  const double* cdf[kMaxModes];
  int64_t I[kMaxModes];
  int npos;                      // N - 1
  const uint64_t* seed_dev;      // if non-null, the Philox key is read from here
  int uniform;                   // uniform sampling (Sec. 5): p and cdf unused
  // fused kernel only: rows from given (merged) samples instead of drawing them, and a
  // device-side row count (rows >= *jdev are not touched)
  const int32_t* given_idx = nullptr;
  const double* given_w = nullptr;
  const int64_t* jdev = nullptr;
};
cudaError_t launch_sample(const SampleArgs& a, int64_t J, uint64_t seed, uint64_t update_id,
                          int32_t* idx, double* w, cudaStream_t st);

struct ChainArgs {
  const double* core[kMaxModes]; // per ring position m, slice-major
  int64_t I[kMaxModes];
  int rl[kMaxModes], rr[kMaxModes];
  int npos;
};
cudaError_t launch_subchain(const ChainArgs& a, const int32_t* idx, const double* w,
                            int64_t J, void* A, bool f64, unsigned* err, cudaStream_t st);

struct GatherArgs {
  int64_t stride[kMaxModes];     // element stride of the mode at ring position m
  int64_t I[kMaxModes];
  int npos;
  int64_t In;                    // length of the gathered mode
  int64_t stride_n;              // its stride
};

// Fused sampler + subchain (+ fibres) of the driver: the same draws as launch_sample, the
// same rows as launch_subchain and, when ga and Y are given, the same fibres as
// launch_gather (in X's dtype x_f64, Y in the rows' dtype), in one launch; p and the CDFs
// are staged in shared memory when they fit.
cudaError_t launch_sample_chain(const SampleArgs& sa, const ChainArgs& ca, int64_t J,
                                uint64_t seed, uint64_t update_id, int32_t* idx, double* w,
                                void* A, bool f64, cudaStream_t st,
                                const GatherArgs* ga = nullptr, const void* X = nullptr,
                                bool x_f64 = false, void* Y = nullptr);
// out = X viewed as [pre][In][post] (row-major) with the middle mode moved last:
// out[a][q][i] = X[a][i][q] (gather.cu). The drivers use it to give a strided mode contiguous
// fibres.
cudaError_t launch_mode_last(const void* X, bool x_f64, int64_t pre, int64_t In, int64_t post,
                             void* out, cudaStream_t st);
cudaError_t launch_gather(const GatherArgs& a, const void* X, bool x_f64, const int32_t* idx,
                          const double* w, int64_t J, void* Y, bool y_f64, unsigned* err,
                          cudaStream_t st);

// Dense TR-ALS (Alg. 1) rows: every multi-index of the modes other than n in row-major order
// (the last mode fastest), written in ring order as idx[P][N-1]; and Y = X_[n]^T with rows
// in that order (Y[r][i], r = pre * P_post + post for X viewed as [P_pre][I_n][P_post]).
struct DenseDims {
  int64_t I[kMaxModes];
};
cudaError_t launch_enumerate(int N, int n, const DenseDims& d, int32_t* idx, cudaStream_t st);
cudaError_t launch_unfold(const void* X, bool x_f64, int N, int n, const DenseDims& d, void* Y,
                          bool y_f64, cudaStream_t st);

// Normal-equation contraction: partial[s][r][c] = sum over the s-th chunk of rows j of
// A[j][r] * [A | Y][j][c], r < L, c < L + I. Returns the number of chunks in *splits.
size_t normal_eq_workspace(int64_t J, int L, int64_t I, bool f64, int* splits);

// The same contraction on the tensor cores (tcgen05, TF32 split into hi + lo, FP32
// accumulation in TMEM) for FP32 inputs; FP32 partials [splits][L][L + I].
size_t normal_eq_tc_workspace(int64_t J, int L, int64_t I, int* splits);
// wait_limit: polls per pipeline wait of the main loop (< 0: the default, 2^26); when a
// wait expires the kernel records kErrTimeout in *err and writes no partials.
// jdev (optional, device): the number of rows actually present (<= J); rows beyond it are
// not read and the partials of chunks beyond it are zero.
cudaError_t launch_normal_eq_tc(const float* A, const float* Y, int64_t J, int L, int64_t I,
                                float* partial, int splits, unsigned* err, cudaStream_t st,
                                long long wait_limit = -1, const int64_t* jdev = nullptr);
cudaError_t launch_normal_eq(const void* A, const void* Y, bool f64, int64_t J, int L,
                             int64_t I, void* partial, int splits, cudaStream_t st,
                             const int64_t* jdev = nullptr);

// Gram of a row-major matrix: trans=false: G = A^T A (cols x cols); trans=true:
// G = A A^T (rows x rows). Partials [splits][n][n] FP64; only tiles on or above the
// diagonal are written (entry (p, q) with p <= q is valid).
size_t gram_workspace(int64_t rows, int cols, bool trans, int* splits);
cudaError_t launch_gram(const double* A, int64_t rows, int cols, int64_t lda, bool trans,
                        double* partial, int splits, cudaStream_t st);
// G = A^T A (trans = false) from double-float planes A = hi + lo (row-major, lda), in
// compensated FP32 arithmetic; same partial layout and split count as launch_gram.
cudaError_t launch_gram_ff(const float* Ah, const float* Al, int64_t rows, int cols,
                           int64_t lda, double* partial, int splits, cudaStream_t st);

// Fixed-order reduction over splits s = 0..splits-1 of an nrows x ncols block of partials
// (row stride pld, split stride pstride; FP32 or FP64) into FP64. Columns c < c_split go
// to out1[r*ld1 + c]; columns c >= c_split go transposed to out2[(c - c_split)*ld2 + r].
// Optional FP32 forms of out1 (an n x n symmetric matrix) for the one-CTA factorisations,
// written by the same reduction: hi (and lo: the double-float split) at [r*lda + c] for
// c >= r (the panel work-array layout), and img (the FP32 image of the whole matrix) at
// [r*np + c]. Null pointers are skipped.
struct ReduceSplit {
  float* hi = nullptr;
  float* lo = nullptr;
  int lda = 0;
  float* img = nullptr;
  int np = 0;
  float* t_hi = nullptr;   // double-float planes of out2 (same layout), for launch_gram_ff
  float* t_lo = nullptr;
};
cudaError_t launch_reduce(const void* partial, bool partial_f32, int splits, int64_t pstride,
                          int64_t pld, int64_t nrows, int64_t ncols, int64_t c_split,
                          double* out1, int64_t ld1, double* out2, int64_t ld2,
                          cudaStream_t st, const ReduceSplit& split = ReduceSplit{});

// Cholesky G = L L^T of the n x n FP64 matrix G (row-major, ld n; only the upper triangle
// G[j][i], j <= i, is read), one CTA. A pivot <= tol_scale * max diag is
//   mode 0 (solve): fatal -> *info = column + 1 and the singular error bit;
//   mode 1 (leverage): the column is dropped (keep = 0) and the factorisation continues.
// Outputs: Lrow (n x n row-major lower factor), Lcol (its transpose), invdiag[n] (1/L_cc,
// 0 for dropped columns), keep[n], *info (0 = success); optionally the padded images read
// by launch_trsm: img64/img32[c*(n+1) + r] = L[r][c] and gimg32[c*(n+1) + r] = G[r][c]
// (buffers of trsm_image_bytes(n, ...) bytes).
// Mixed-precision LS step: an FP32 factor when every pivot > tol32 * max diag, written as the
// FP32 image img32 + invdiag + keep + info; otherwise the FP64 factorisation with tol64
// and the mode's rule (as launch_cholesky: 0 stops, 1 drops the column).
// With wimg and fast (and pre, 4 <= n <= 128) an FP32 factor and its inverse are first formed
// together in one CTA (chol_inv.cuh): on success W = L_f^-1 goes to wimg (the image
// launch_solve_inv reads), keep = 1, *info = 0 and *fast = 1, and the launches above exit at
// once; otherwise *fast = 0 and they run as described. Pass the same fast to launch_solve_inv.
cudaError_t launch_cholesky_mixed(const double* G, int n, int mode, double tol64, double tol32,
                                  double* Lrow, double* Lcol, double* invdiag, int* keep,
                                  int* info, unsigned* err, cudaStream_t st, float* img32,
                                  float* gimg32, const float* pre = nullptr,
                                  float* wimg = nullptr, int* fast = nullptr);
// Mixed-precision drivers' leverage Gram of a tall matrix (mode 1): double-float factor when
// every pivot > tolff * max diag (FP64 image img64 + invdiag + keep + info), otherwise the FP64
// factorisation with tol64 and column dropping (as launch_cholesky, mode 1).
cudaError_t launch_cholesky_lev_mixed(const double* G, int n, double tol64, double tolff,
                                      double* Lrow, double* Lcol, double* invdiag, int* keep,
                                      int* info, unsigned* err, cudaStream_t st, double* img64,
                                      const float* pre_hi = nullptr,
                                      const float* pre_lo = nullptr,
                                      const int* run_if = nullptr);
// pre / pre_hi, pre_lo: the work array's planes already written by launch_reduce (a
// ReduceSplit with lda = (n + 3) & ~3), or null to convert from G.
// After launch_cholesky_lev_mixed: img64 = hi + lo of the FP32 planes it left in Lrow / Lcol
// when its double-float branch succeeded (*info == 2); otherwise nothing.
// run_if (both launches, optional): nothing is done unless *run_if != 0.
cudaError_t launch_ff_image(const double* Lrow, const double* Lcol, int n, const int* info,
                            double* img64, cudaStream_t st, const int* run_if = nullptr);
cudaError_t launch_cholesky(const double* G, int n, int mode, double tol_scale, double* Lrow,
                            double* Lcol, double* invdiag, int* keep, int* info,
                            unsigned* err, cudaStream_t st, double* img64 = nullptr,
                            float* img32 = nullptr, float* gimg32 = nullptr);

// Triangular solves with the factor of launch_cholesky for nvec vectors (row v of rhs,
// leading dimension ld, length n):
//   mode 0: ell[v] = || L^-1 rhs_v ||^2 (leverage rows);
//   mode 1: z = L^-T L^-1 rhs_v written to core_out[v][a][b] = z[a + Rl*b];
//   mode 2: as mode 1 plus one refinement step z += M^-1 (rhs_v - M z), M (n x n FP64).
// f32 selects FP32 arithmetic (factor and M rounded to FP32), else FP64. Nothing is done
// when *info != 0 (info may be NULL).
// Limg: padded factor image in the arithmetic type (FP32 when f32, else FP64), Mimg: FP32
// image of M (mode 2, f32); both optional (NULL: converted from Lcol / M instead).
// cdf (mode 0, optional): the CTA that finishes last forms p = ell / sum(ell) and the CDF
// (fixed-order scan); *counter must be 0 before the launch and is 0 again after it; when
// skip && *skip != 0 p and the CDF are left unchanged.
struct CdfEpilogue {
  unsigned* counter;
  double* p;
  double* cdf;
  const int* skip;
  unsigned* err;
  const int* run_if = nullptr;   // when given, the launch does nothing unless *run_if != 0
};
cudaError_t launch_trsm(int mode, bool f32, int n, const double* Lrow, const double* Lcol,
                        const double* invdiag, const int* info, int64_t nvec, const double* rhs,
                        int64_t ld, const double* M, int Rl, int Rr, double* core_out,
                        double* ell, cudaStream_t st, const void* Limg = nullptr,
                        const float* Mimg = nullptr, const CdfEpilogue* cdf = nullptr);
size_t trsm_image_bytes(int n, bool f32);

// Leverage scores (and, unless skip && *skip, p and the CDF) of the rows of a wide I x L
// row-major FP64 matrix (row stride lda) by one-sided Jacobi in one CTA (jacobi.cu): the rank
// rule of a singular value decomposition, sigma > max(I, L) * eps * sigma_max. For
// 1 <= I < L with I <= kJacobiMaxI; a zero matrix records kErrSingular and gives the
// uniform distribution.
constexpr int kJacobiMaxI = 48;
constexpr size_t kJacobiSmem = 200 * 1024;
bool leverage_jacobi_fits(int64_t I, int L);
cudaError_t launch_leverage_jacobi(const double* A, int64_t I, int L, int64_t lda, double* ell,
                                   double* p, double* cdf, const int* skip, unsigned* err,
                                   cudaStream_t st);

// Mixed-precision LS solve for L <= 128 (solve_inv.cu): W = L_f^-1 from the factor's FP32
// image (into Wimg, trsm_image_bytes(n, true) bytes), then z = W^T W b, r = b - M z,
// z += W^T W r for every row b of rhs (ld), written as the new core; nothing when *info != 0.
// With fast (launch_cholesky_mixed's flag) W is not formed when *fast != 0: it is already in Wimg.
bool solve_inv_fits(int n);
cudaError_t launch_solve_inv(int n, const float* Limg, const float* Mimg,
                             const double* invdiag, const int* info, int64_t nvec,
                             const double* rhs, int64_t ld, int Rl, int Rr, double* core_out,
                             float* Wimg, cudaStream_t st, const int* fast = nullptr);

// The mixed drivers' leverage scores of a tall I x n row-major matrix A given as double-float
// planes (Ah + Al, row stride lda), 4 <= n <= 128 (lev_precond.cu): an FP32 Cholesky factor of
// K = A^T A (from the reduction's FP32 work array K_hi, row stride lda_k) and its inverse X
// as preconditioner, C = X K X^T = I + E in double-float from K's planes, and
// ell_i = w_i^T (I + E)^-1 w_i with w_i = X a_i by a short series; then, from the last CTA,
// p and the CDF as launch_trsm's epilogue (ep.counter 0 before the launch). When the FP32
// factorisation fails or ||E||_F is too large for the series, nothing is written and
// *state = 1 (0 otherwise): the caller's fallback launches are gated on it (run_if).
// Four launches, issued in order by stage = 0 (FP32 factor and its inverse X in one CTA;
// sets *state), 1 (U = X K), 2 (E = U X^T - I), 3 (rows, p and the CDF; reads ep.skip);
// lda_k must be (n + 3) & ~3.
struct LevPrecond {
  const float* K_hi;
  const float* K_lo;
  int lda_k;
  float* Ximg;       // X = L^-1, padded FP32 image (trsm_image_bytes(n, true) bytes)
  float* Uh;         // U = X K as double-float planes, n x lda_k each
  float* Ul;
  float* E;          // n x lda_k
  float* esq;        // lev_precond_ctas(n)
  int* state;
  float* gph;        // launch_gram_dd scratch (gram_dd_partial_floats each)
  float* gpl;
  float tau = 1e-2f; // largest ||E||_F of the series (above it: the fallback)
};
bool lev_precond_fits(int64_t I, int n);
// K = A^T A of the tall I x n double-float planes (row stride lda_a) in one launch: K's
// double-float planes kh/kl[r*lda + c] (c >= r) and K in FP64 (k64, n x n). Scratch: ph and pl
// of gram_dd_partial_floats(I, n) floats each, and cnt[ntiles] zero on entry (left zero).
size_t gram_dd_partial_floats(int64_t I, int n);
cudaError_t launch_gram_dd(const float* Ah, const float* Al, int64_t I, int n, int64_t lda_a,
                           float* ph, float* pl, unsigned* cnt, float* kh, float* kl, int lda,
                           double* k64, cudaStream_t st);
int lev_precond_ctas(int n);
cudaError_t launch_lev_precond(int stage, const LevPrecond& lp, int n, int64_t I,
                               const float* Ah, const float* Al, int64_t lda, double* ell,
                               const CdfEpilogue& ep, cudaStream_t st);

// dst[e] = hi[e] + lo[e] in FP64 (lev_precond.cu).
cudaError_t launch_planes_sum(const float* hi, const float* lo, int64_t count, double* dst,
                              cudaStream_t st);
// *dst = src ? *src : v, on the stream (lev_precond.cu).
cudaError_t launch_copy_int(const int* src, int v, int* dst, cudaStream_t st);

// Merging repeated draws (merge.cu; Sec. 4.2): idx_out / w_out receive one row per distinct
// multi-index in the order of first occurrence, weight w * sqrt(count), and *J_out (device)
// their number. For J <= kMergeMaxJ and prod of the sampled sizes < 2^63 (merge_fits, which
// also fills the ring linear-index strides).
constexpr int kMergeMaxJ = 8192;
struct MergeArgs {
  uint64_t stride[kMaxModes];
  int Jpow2;
};
bool merge_fits(int64_t J, int npos, const int64_t* I, MergeArgs* a);
cudaError_t launch_merge(const int32_t* idx, const double* w, int64_t J, int npos,
                         const MergeArgs& a, int32_t* idx_out, double* w_out, int64_t* J_out,
                         cudaStream_t st);

// Core initialisation N(0,1) by Philox + Box-Muller.
cudaError_t launch_init_normal(double* out, int64_t count, uint64_t seed, uint32_t stream_id,
                               const uint64_t* seed_dev, cudaStream_t st);

// Number of SMs of the current device (queried once per device and cached); grids of the
// streaming kernels and the split counts of the contractions are sized from it.
int sm_count();

// Raise the dynamic shared-memory limit of the kernels that need it (once per device);
// on failure *which names the kernel.
cudaError_t init_kernel_attributes(const char** which);

// Fit: partial sums of squares of (X - TR) and X over blocks; FP64 outputs [2][blocks].
struct FitArgs {
  const double* core[kMaxModes];  // slice-major, natural mode order
  int64_t dims[kMaxModes];
  int ranks[kMaxModes];
  int N;
};
// Workspace: 2 * blocks partial sums, then the right factors of the mode split.
size_t fit_workspace(const FitArgs& a, bool x_f64, int* blocks);
cudaError_t launch_fit(const FitArgs& a, const void* X, bool x_f64, void* ws, int blocks,
                       unsigned* err, cudaStream_t st);

}  // namespace trk
