/*
 * trals.h -- C ABI of libtrals.so, a GB300 (sm_103a) implementation of the hot path of
 * TR-ALS-Sampled (Malik & Becker, "A Sampling-Based Method for Tensor Ring
 * Decomposition", ICML 2021, Alg. 2 with Alg. 3 and Alg. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Modes are 0-based: k = 0..N-1. ranks[k] is the paper's R_{k+1}; core k has left rank
 *    Rl_k = ranks[(k-1+N) % N] and right rank Rr_k = ranks[k] (the paper's
 *    G^(k+1) in R^{R_k x I_{k+1} x R_{k+1}}, Sec. 3.1, eq. 1).
 *  - Cores are FP64, slice-major: core_k[i][a][b] at offset (i*Rl_k + a)*Rr_k + b, so the
 *    lateral slice G(:, i, :) is one contiguous Rl_k x Rr_k row-major block.
 *  - X is dense, row-major (last mode fastest), FP32 or FP64.
 *  - Sampled multi-indices idx[J][N-1] (int32) are in ring order: position m holds the
 *    index of mode (k+1+m) % N (Def. 2 / Alg. 3).
 *  - Design rows: row j, column c = a + Rl_k*b holds the (b, a) entry of the Rr_k x Rl_k
 *    slice product of Alg. 4 (the paper's column overline{r_{k-1} r_k}).
 *  - All tensor arguments are DEVICE pointers owned by the caller unless stated; arrays of
 *    per-mode pointers (cores, p, cdf) and dims/ranks are HOST arrays.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and returns a status; nothing aborts or traps. Argument errors are reported
 *    before any launch. Errors found on the device (a non-positive Cholesky pivot, an
 *    out-of-range caller index) are recorded in the context and returned by the next
 *    tr_status_sync() (or by the synchronous tr_als_sampled / tr_rel_error).
 *  - A context owns only its device workspace (grown on demand, capped by the HBM budget
 *    given at creation). Calls that share a context must not overlap in time: issue them
 *    on one stream.
 */
#ifndef TRALS_H
#define TRALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tr_status {
  TR_OK = 0,
  TR_ERR_INVALID_ARG = 1,  /* bad sizes, null pointers, unsupported rank/mode count     */
  TR_ERR_OOM = 2,          /* device allocation failed                                  */
  TR_ERR_BUDGET = 3,       /* workspace would exceed the context's HBM budget          */
  TR_ERR_SINGULAR = 4,     /* non-positive pivot in the normal equations, or zero core */
  TR_ERR_TIMEOUT = 5,      /* a bounded device wait expired (tensor-core pipeline; see  */
                           /* tr_set_wait_limit), or tr_server_wait's time ran out     */
  TR_ERR_CUDA = 6,         /* a CUDA runtime call failed (see tr_last_error)            */
  TR_ERR_NOT_CONVERGED = 7 /* a served request stopped at its sweep cap (result kept)    */
} tr_status;

typedef enum tr_dtype { TR_F32 = 0, TR_F64 = 1 } tr_dtype;

/* Arithmetic of the least-squares step (rows a3-a6) and of the drivers' distributions.
 * TR_PREC_FP64 : design rows, fibres, contractions, Cholesky and solves in FP64.
 * TR_PREC_MIXED: design rows and fibres in FP32, contractions with FP32 accumulation.
 *                The normal matrix is factored in FP32 when every pivot exceeds
 *                L*eps32*max diag, else in FP64 (same singular rule as TR_PREC_FP64);
 *                FP32 solves (for L <= 128 products by the factor's FP32 inverse, formed
 *                together with the FP32 factor in one pass; triangular substitutions
 *                otherwise) and one step of iterative refinement against the
 *                FP32-accurate normal-equation residual. In the drivers, the leverage
 *                scores of a tall matrix (I >= L, 4 <= L <= 128) are those of
 *                tr_leverage_planes: an FP32 Cholesky preconditioner of the double-float
 *                Gram and a double-float series, or, when that preconditioner is poor, the
 *                Gram factored in double-float (pairs of FP32, about 46 significant bits)
 *                when every pivot exceeds max(I,L)*2^-40*max diag, else in FP64 with column
 *                dropping. All other leverage arithmetic, and tr_leverage, is FP64.
 *                The drivers (both precisions) read the fibres of a strided mode from a
 *                copy of X with that mode last, made at the start of each call, when the
 *                scattered reads would move more bytes than the copy and memory allows;
 *                results are bitwise the same as reading X itself. */
typedef enum tr_precision { TR_PREC_FP64 = 0, TR_PREC_MIXED = 1 } tr_precision;

/* How tr_als_sampled, tr_als_sampled_host and tr_als_sampled_batched draw their samples.
 * TR_SAMPLING_LEVERAGE: Alg. 2 as stated -- products of the cores' leverage-score
 *                       distributions (Alg. 3), each refreshed after its core's update.
 * TR_SAMPLING_UNIFORM : the uniform variant of Sec. 5 (draws as tr_sample_uniform); no
 *                       distribution is ever formed, so the leverage stages are skipped. */
typedef enum tr_sampling { TR_SAMPLING_LEVERAGE = 0, TR_SAMPLING_UNIFORM = 1 } tr_sampling;

typedef struct tr_ctx tr_ctx;
typedef void* tr_stream;

#define TR_MAX_MODES 16   /* largest N                                   */
#define TR_MAX_RANK_PRODUCT 256 /* largest Rl_k * Rr_k (LS unknowns per row) */

/* Create a context on CUDA device `device`. hbm_budget_bytes caps the workspace the
 * context may allocate (0 = no cap). *ctx receives the handle (NULL on failure). */
tr_status tr_create(tr_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Free the context and its workspace (synchronises the device first). NULL is a no-op. */
void tr_destroy(tr_ctx* ctx);

/* Text of the last error reported by a call on this context ("" if none); with ctx NULL,
 * the reason of the last failed tr_create or tr_solve_noalloc. */
const char* tr_last_error(const tr_ctx* ctx);

/* Wait for `stream`, then return and clear the device-side error record of the context
 * (TR_ERR_TIMEOUT for an expired bounded wait, TR_ERR_INVALID_ARG for out-of-range sample
 * indices, TR_ERR_SINGULAR, or TR_OK; the first that applies in this order). */
tr_status tr_status_sync(tr_ctx* ctx, tr_stream stream);

/* Row a1 -- sampling distribution of one core (Def. 4; eq. for p^(n); Alg. 2, "compute
 * distributions" and "update n-th distribution").
 * core  : FP64 [I][Rl][Rr]; the matrix G_(2) is I x (Rl*Rr).
 * p     : FP64 [I] out, p[i] = ell_i(G_(2)) / sum_i ell_i(G_(2)).
 * cdf   : FP64 [I] out, inclusive prefix sum of p in index order.
 * Leverage scores, in FP64: for a wide G_(2) with few rows (I < L = Rl*Rr, I <= 48) by
 * one-sided Jacobi rotations of its rows, keeping the directions whose singular value is
 * above max(I,L)*eps*sigma_max (the rule of a singular value decomposition); otherwise from
 * a Cholesky-based thin QR of G_(2) (or of G_(2)^T when I < L), with dependent columns
 * dropped at pivot <= max(I,L)*eps*max diag, which resolves singular values down to about
 * sqrt(max(I,L)*eps)*sigma_max. The drivers form every distribution the same way.
 * A zero core records TR_ERR_SINGULAR and yields the uniform distribution. */
tr_status tr_leverage(tr_ctx* ctx, const double* core, int64_t I, int Rl, int Rr,
                      double* p, double* cdf, tr_stream stream);

/* Row a1 as the mixed-precision drivers compute it after each update (Def. 4; eq. for
 * p^(n); Alg. 2, "update n-th distribution"): the distribution of a tall matrix A
 * (I >= L, 4 <= L <= 128) given as two FP32 planes, A = A_hi + A_lo (row-major I x L), the
 * form in which the drivers hold B^T. K = A^T A is formed in double-float; an FP32 Cholesky
 * factor of K and its inverse X precondition it, C = X K X^T = I + E is formed in
 * double-float, and ell_i = w_i^T (I + E)^-1 w_i with w_i = X a_i by the series
 * sum_k (-E)^k, taken through E^4 (||E||_F <= 1e-3) or E^6 (||E||_F <= 1e-2). If the FP32
 * factorisation meets a pivot <= L*eps32*max diag or ||E||_F > 1e-2, the double-float
 * factorisation of K with FP64 fallback and FP64 row solves is used instead (the rank rule of
 * TR_PREC_MIXED above). Both branches run on the device with no host round trip.
 * A_hi, A_lo : device FP32 [I][L] (16-byte aligned).
 * p, cdf     : device FP64 [I] out, as tr_leverage.
 * branch     : optional device int out: 0 when the preconditioned form was used, 1 when
 *              the factorisation fallback was.
 * Other shapes return TR_ERR_INVALID_ARG. */
tr_status tr_leverage_planes(tr_ctx* ctx, const float* A_hi, const float* A_lo, int64_t I,
                             int L, double* p, double* cdf, int* branch, tr_stream stream);

/* Row a2 -- J i.i.d. draws from q^{!=k} = prod_{j!=k} p^(j) (Alg. 3; Def. 5).
 * p, cdf   : host arrays of N device pointers (entry k unused), FP64 [dims[j]].
 * seed, update_id : Philox4x32-10 key and counter words: the uniform for sample j at ring
 *            position m comes from counter (j, m/2, update_id lo, update_id hi), words
 *            (2(m%2), 2(m%2)+1) as (hi, lo), u = top 53 bits * 2^-53.
 * idx      : int32 [J][N-1] out (ring order); index = smallest i with u < cdf[i], or
 *            the largest i with p[i] > 0 when u >= cdf[last].
 * w        : FP64 [J] out, w_j = 1 / sqrt(J * prod_m p(idx[j][m])) (product in ring
 *            order). */
tr_status tr_sample(tr_ctx* ctx, int N, int k, const int64_t* dims,
                    const double* const* p, const double* const* cdf, int64_t J,
                    uint64_t seed, uint64_t update_id, int32_t* idx, double* w,
                    tr_stream stream);

/* Row a2, uniform variant -- J i.i.d. draws from the uniform distribution
 * q^{!=k} = 1 / prod_{j!=k} I_j, the alternative to leverage-score sampling that Sec. 5
 * evaluates (uniform sampling experiment); no distribution is read.
 * seed, update_id : as for tr_sample: the same Philox uniform u per (sample, position).
 * idx      : int32 [J][N-1] out (ring order); index = floor(u * I) in FP64, clamped to I-1.
 * w        : FP64 [J] out, every entry sqrt(P / J), P = prod of the sampled modes' sizes
 *            formed in FP64 in ring order (= 1 / sqrt(J q) of Def. 5). */
tr_status tr_sample_uniform(tr_ctx* ctx, int N, int k, const int64_t* dims, int64_t J,
                            uint64_t seed, uint64_t update_id, int32_t* idx, double* w,
                            tr_stream stream);

/* Row a3 -- sampled subchain S G_[2]^{!=k} (Alg. 4; Def. 3).
 * cores : host array of N device pointers (entry k unused), FP64 slice-major.
 * idx   : int32 [J][N-1] ring order; w: FP64 [J] row scales (NULL = 1).
 * A     : [J][Rl_k*Rr_k] out in A_dtype (TR_F32: products in FP32; TR_F64: in FP64).
 * Out-of-range indices record TR_ERR_INVALID_ARG and give zero rows. */
tr_status tr_subchain(tr_ctx* ctx, int N, int k, const int64_t* dims, const int* ranks,
                      const double* const* cores, const int32_t* idx, const double* w,
                      int64_t J, void* A, tr_dtype A_dtype, tr_stream stream);

/* Row a4 -- sampled fibres S X_[k]^T (Alg. 2, "compute X~"; Def. 2).
 * X : dense row-major [dims[0]]...[dims[N-1]] in X_dtype.
 * Y : [J][dims[k]] out in Y_dtype, Y[j][i] = w_j * X(.., i at mode k, ..).
 * w : FP64 [J] (NULL = 1). Out-of-range indices record TR_ERR_INVALID_ARG, zero rows. */
tr_status tr_gather(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N,
                    const int64_t* dims, int k, const int32_t* idx, const double* w,
                    int64_t J, void* Y, tr_dtype Y_dtype, tr_stream stream);

/* Rows a5 + a6 -- solve the sampled LS argmin_Z || A Z - Y ||_F (Alg. 2, LS step) through
 * the normal equations M = A^T A, B = A^T Y, Cholesky M = L L^T (FP64, or FP32 as
 * tr_precision describes), Z = M^-1 B (and, in TR_PREC_MIXED, one refinement
 * Z += M^-1 (B - M Z)), then write the new core
 * core_out[i][a][b] = Z[a + Rl*b][i].
 * A : [J][Rl*Rr], Y : [J][I], both in `dtype` (TR_F32 for TR_PREC_MIXED, TR_F64 for
 * TR_PREC_FP64). A pivot <= L*eps*max diag(M) records TR_ERR_SINGULAR and leaves
 * core_out unchanged. */
tr_status tr_solve(tr_ctx* ctx, const void* A, const void* Y, tr_dtype dtype, int64_t J,
                   int Rl, int Rr, int64_t I, tr_precision prec, double* core_out,
                   tr_stream stream);

/* The whole method (Alg. 2) with a fixed number of sweeps, synchronous.
 * X          : device, row-major, X_dtype.
 * init_cores : host array of N device pointers with the initial cores (entry 0 unused),
 *              or NULL: cores 1..N-1 are drawn i.i.d. N(0,1) on the device from `seed`.
 * cores      : host array of N device pointers, FP64 slice-major, receive the result.
 * Sweep s, core n draws its samples with update_id = s*N + n.
 * prec       : TR_PREC_MIXED expects X in FP32 or FP64; TR_PREC_FP64 any.
 * Returns TR_ERR_SINGULAR if any update met a singular normal matrix (that core kept). */
tr_status tr_als_sampled(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N,
                         const int64_t* dims, const int* ranks, int64_t J, int sweeps,
                         uint64_t seed, tr_precision prec, const double* const* init_cores,
                         double* const* cores, tr_stream stream);

/* tr_als_sampled with one sample size per sweep (Sec. 4.2: J can be changed at any point
 * at no cost): sweep s draws J_per_sweep[s] samples per update (host array of `sweeps`
 * entries, each in [1, 2^31-1]); the workspace is sized for the largest. Everything else
 * as tr_als_sampled. */
tr_status tr_als_sampled_schedule(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N,
                                  const int64_t* dims, const int* ranks,
                                  const int64_t* J_per_sweep, int sweeps, uint64_t seed,
                                  tr_precision prec, const double* const* init_cores,
                                  double* const* cores, tr_stream stream);

/* tr_als_sampled with one sample size per core update (Sec. 4.2: J can be changed at any
 * point at no cost): the update of core n in sweep s draws J_per_update[s*N + n] samples
 * (host array of sweeps*N entries, each in [1, 2^31-1]); the workspace is sized for the
 * largest. Everything else as tr_als_sampled. */
tr_status tr_als_sampled_adaptive(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N,
                                  const int64_t* dims, const int* ranks,
                                  const int64_t* J_per_update, int sweeps, uint64_t seed,
                                  tr_precision prec, const double* const* init_cores,
                                  double* const* cores, tr_stream stream);

/* Merging repeated draws (Sec. 4.2). Draws are made with replacement, so a multi-index can
 * be drawn several times; its rows of the sketch are then identical and carry the same
 * weight w (Def. 5), and c copies of a row contribute to the normal equations what one row
 * with weight sqrt(c) * w contributes.
 * tr_merge_samples: idx [J][N-1], w [J] (device, as tr_sample writes them) -> idx_out, w_out
 *   (device, capacity J) with one row per distinct multi-index, in the order of first
 *   occurrence, weight w * sqrt(count); *J_out (device int64) receives their number. Rows
 *   of idx_out / w_out beyond *J_out are not written. J must be in [1, 8192] and the product
 *   of the sampled modes' sizes below 2^63, else TR_ERR_INVALID_ARG before any launch.
 * tr_set_merge_duplicates(ctx, 1): the single-problem drivers of this context merge every
 *   update's draws before forming rows and fibres (updates with J above 8192 or an index
 *   space of 2^63 or more are not merged); the rows, fibres and contraction then run over the
 *   merged count only. Results equal the unmerged ones up to rounding. Off by default. */
tr_status tr_merge_samples(tr_ctx* ctx, int N, int k, const int64_t* dims, const int32_t* idx,
                           const double* w, int64_t J, int32_t* idx_out, double* w_out,
                           int64_t* J_out, tr_stream stream);
tr_status tr_set_merge_duplicates(tr_ctx* ctx, int on);
tr_status tr_get_merge_duplicates(const tr_ctx* ctx, int* on);

/* Dense TR-ALS (Alg. 1), the comparison method of Sec. 5, with a fixed number of sweeps,
 * synchronous. Core update n solves the full least-squares problem
 * argmin_Z || G_[2]^{!=n} Z - X_[n]^T ||_F over all prod_{j!=n} I_j rows, each with weight 1
 * (Def. 5 with S = I), through the same normal-equation path as tr_als_sampled (rows a3,
 * a5, a6; same tr_precision arithmetic). No distribution is formed. Arguments as
 * tr_als_sampled, without J (seed only draws the initial cores when init_cores is NULL).
 * Workspace: about prod I * es + max_n prod_{j!=n} I_j * (L_max * es + 4 (N-1)) bytes plus
 * the LS step's, es = 4 (TR_PREC_MIXED) or 8. Every dims[k] must be <= 2097120. */
tr_status tr_als(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N, const int64_t* dims,
                 const int* ranks, int sweeps, uint64_t seed, tr_precision prec,
                 const double* const* init_cores, double* const* cores, tr_stream stream);

/* Same as tr_als_sampled with X and the cores in HOST memory: X is copied to the device,
 * the method runs, and the cores are copied back into the host arrays cores_host[k]
 * (FP64 slice-major). init_cores_host may be NULL. Pinned host memory is fastest. */
tr_status tr_als_sampled_host(tr_ctx* ctx, const void* X_host, tr_dtype X_dtype, int N,
                              const int64_t* dims, const int* ranks, int64_t J, int sweeps,
                              uint64_t seed, tr_precision prec,
                              const double* const* init_cores_host,
                              double* const* cores_host, tr_stream stream);

/* Relative error ||TR(cores) - X||_F / ||X||_F (Sec. 5.1), synchronous; *rel_err is a
 * host double. Reconstruction runs in X's precision with FP64 sums of squares. */
tr_status tr_rel_error(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N,
                       const int64_t* dims, const int* ranks, const double* const* cores,
                       double* rel_err, tr_stream stream);

/* Draw cores i.i.d. N(0,1) (Philox4x32-10 + Box-Muller) into the device buffers cores[k],
 * k in [k_begin, N). Used by tr_als_sampled when init_cores is NULL. */
tr_status tr_init_cores(tr_ctx* ctx, int N, const int64_t* dims, const int* ranks,
                        uint64_t seed, int k_begin, double* const* cores, tr_stream stream);

/* One independent problem of a batch (see tr_als_sampled_batched). */
typedef struct tr_instance {
  const void* X;                   /* device, row-major [dims[0]]...[dims[N-1]]            */
  int N;                           /* number of modes, 2..TR_MAX_MODES                      */
  int64_t dims[TR_MAX_MODES];
  int ranks[TR_MAX_MODES];         /* ranks[k] = paper's R_{k+1}, each in [1, 16]          */
  int64_t J;                       /* samples per least-squares problem                     */
  uint64_t seed;                   /* Philox key of this instance's draws (and its init)    */
  double* cores[TR_MAX_MODES];     /* device FP64 slice-major [I_k][Rl_k][Rr_k], results   */
  int init_given;                  /* nonzero: cores[1..N-1] already hold the initial cores */
} tr_instance;

/* Alg. 2 for `count` independent problems at once, synchronous. Every stage of every
 * sweep is one launch for all instances (one CTA or a few per instance), so many small
 * problems fill the GPU together. Each instance performs sweeps * N updates with the
 * same draws, sizes and arithmetic as tr_als_sampled on that instance alone would with
 * the same precision, except that the normal equations are summed in one fixed order per
 * instance (no split over the samples); its results do not depend on the other instances
 * of the batch. All instances share X_dtype and prec. The sequence of launches is
 * captured once per batch geometry as a CUDA graph and replayed.
 * Returns TR_ERR_SINGULAR if any update of any instance met a singular normal matrix
 * (that core kept). */
tr_status tr_als_sampled_batched(tr_ctx* ctx, const tr_instance* inst, int count,
                                 tr_dtype X_dtype, int sweeps, tr_precision prec,
                                 tr_stream stream);

/* What the LS step (tr_solve and every driver of the context) does with a pivot of the
 * normal matrix <= L*eps*max diag (FP64 rule; the mixed path applies it on its FP64
 * branch):
 * TR_LS_RANK_STOP : record TR_ERR_SINGULAR and keep the core (the default);
 * TR_LS_RANK_DROP : drop that column -- its unknowns are 0 and it updates nothing -- and
 *                   solve for the rest: a basic least-squares solution of a rank-deficient
 *                   design, as a QR-based solve returns (the paper's LS step is QR-based).
 *                   TR_PREC_MIXED drops at L*eps32*max diag, the resolution of its FP32
 *                   triangular solves.
 * Other values return TR_ERR_INVALID_ARG. */
typedef enum tr_ls_rank { TR_LS_RANK_STOP = 0, TR_LS_RANK_DROP = 1 } tr_ls_rank;
tr_status tr_set_ls_rank(tr_ctx* ctx, tr_ls_rank rule);
tr_status tr_get_ls_rank(const tr_ctx* ctx, tr_ls_rank* rule);

/* Sampling of the context's driver calls (a context starts with TR_SAMPLING_LEVERAGE).
 * Other values return TR_ERR_INVALID_ARG. */
tr_status tr_set_sampling(tr_ctx* ctx, tr_sampling sampling);
tr_status tr_get_sampling(const tr_ctx* ctx, tr_sampling* sampling);

/* Factorisations of the mixed-precision path (TR_PREC_MIXED) in tr_solve and the drivers:
 * TR_FACTOR_DEFAULT: as TR_PREC_MIXED describes (FP32 normal-matrix factor and double-float
 *                    leverage factor, each with its FP64 fallback);
 * TR_FACTOR_FP64   : both factored in FP64 (the normal matrix with the FP64 singular rule,
 *                    then FP32 triangular solves with one refinement step; the leverage
 *                    Gram as TR_PREC_FP64 does).
 * The batched driver and the server keep their own rules. Other values return
 * TR_ERR_INVALID_ARG. */
typedef enum tr_factorization { TR_FACTOR_DEFAULT = 0, TR_FACTOR_FP64 = 1 } tr_factorization;
tr_status tr_set_factorization(tr_ctx* ctx, tr_factorization f);
tr_status tr_get_factorization(const tr_ctx* ctx, tr_factorization* f);

/* Poll limit of the bounded device waits of this context's tensor-core contraction (rows
 * a5: the pipeline waits of the FP32 normal-equation kernel used by tr_solve and the drivers
 * with TR_PREC_MIXED). A context starts with the default (polls < 0), 2^26 polls per wait,
 * which only a stalled GPU exhausts. When a wait expires the kernel stops issuing, waits for
 * the MMAs it has already committed (with the default limit), frees its tensor memory and
 * returns without writing its partial sums; the LS step then leaves the core unchanged and
 * the next tr_status_sync (or the synchronous driver) returns TR_ERR_TIMEOUT. The context
 * stays usable. polls = 0 makes every such wait expire at once, a diagnostic setting with
 * which a caller or a test can exercise the error path. */
tr_status tr_set_wait_limit(tr_ctx* ctx, int64_t polls);
tr_status tr_get_wait_limit(const tr_ctx* ctx, int64_t* polls);

/* Launch shapes of the batched driver's kernels, chosen per batch geometry by the
 * project's autotuner (paper_2010_08581_gb300/autotune.py), which times the candidates on
 * scratch copies of a batch. Neither field changes any result: samples are independent,
 * and every entry of the normal equations is summed over the samples in the same order
 * for either tile.
 *   samples_per_warp : samples drawn and formed by one warp of the sampling kernel, 1..8
 *   contract_tile    : output tile (64 or 32 square) of the normal-equation contraction
 * A context starts with {4, 64}. tr_set_batched_tiles returns TR_ERR_INVALID_ARG for
 * other values. */
typedef struct tr_batched_tiles {
  int samples_per_warp;
  int contract_tile;
} tr_batched_tiles;

tr_status tr_set_batched_tiles(tr_ctx* ctx, const tr_batched_tiles* tiles);
tr_status tr_get_batched_tiles(const tr_ctx* ctx, tr_batched_tiles* tiles);

/* Least-squares step without any device allocation (the paper has no counterpart; this
 * is a deployment variant of tr_solve).
 *
 * Some callers cannot call cudaMalloc: plug-ins and callbacks that run inside a host
 * framework which owns the device memory and forbids them to allocate, latency-critical
 * serving loops where cudaMalloc/cudaFree would synchronise the device, and hosts that have
 * partitioned all device memory up front. tr_solve_noalloc computes what tr_solve computes
 * on a context with the default settings (TR_LS_RANK_STOP, the default wait limit): the
 * same kernels with the same arguments, so the new core is bit-identical. It takes its
 * scratch from one fixed 16 MiB array that the library keeps in device memory, calls no
 * cudaMalloc, cudaFree or allocating library routine, and needs no context.
 *
 * - Every GPU on which the library is loaded holds the 16 MiB array until the process
 *   exits.
 * - A problem whose scratch (the split partials of the L x (L+I) contraction, the L x I
 *   right-hand sides, the factor and its images) exceeds 16 MiB is rejected with
 *   TR_ERR_INVALID_ARG and a message (tr_last_error(NULL)); nothing is launched. For
 *   J = 4000, L = 100, I = 500 about 7 MiB are used.
 * - All calls share the array and it keeps the previous call's contents (each call clears
 *   what must start at zero), so calls that overlap on the GPU (on different streams, or on
 *   several host threads) race and give wrong results: serialise them on one stream.
 * - The first call on each device (with that device current) resolves the array's
 *   device address and sets kernel attributes; make that first call before any stream
 *   capture begins. The address is kept for the life of the process: after
 *   cudaDeviceReset on that device the entry point must not be called again.
 * - info (device int32, may be NULL) receives 0 on success, column+1 of the first
 *   non-positive pivot, or -1 when a bounded wait of the tensor-core contraction expired
 *   (TR_PREC_MIXED); in both failure cases core_out is left unchanged.
 * Arguments otherwise as tr_solve; the current device must be the one holding the data. */
tr_status tr_solve_noalloc(const void* A, const void* Y, tr_dtype dtype, int64_t J, int Rl,
                           int Rr, int64_t I, tr_precision prec, double* core_out,
                           int32_t* info, tr_stream stream);

/* ------------------------------------------------------------------------------------
 * Serving: continuous batching of independent decompositions (Alg. 2 per request, run
 * until the relative fit 1 - ||TR - X||_F / ||X||_F changes by less than a tolerance from
 * one sweep to the next, one of the stopping criteria of Sec. 4.1).
 *
 * A server owns a slot table, a device workspace arena and a set of CUDA graphs. Each
 * "tick" replays one graph over all occupied slots: one core update per running request
 * (or, for a newly admitted request, the initial distribution of one core), the exact fit of
 * every request that completed a sweep, and the stop rule, all on the device. Requests that
 * arrive while others run are admitted, in submission order, as soon as a slot, arena space
 * and HBM budget are free, and join at the next tick; finished requests release theirs at
 * the end of a tick. A request's result does not depend on which other requests share its
 * ticks: every launch gives each slot its own CTAs and the launch geometry is fixed by the
 * server configuration. With the same configuration, a request's cores after s sweeps equal
 * those of tr_als_sampled_batched with `sweeps` = s on that request alone.
 * ------------------------------------------------------------------------------------ */
#define TR_MAX_SERVED_SWEEPS 64

typedef struct tr_server tr_server;

typedef struct tr_server_config {
  int device;                 /* CUDA device ordinal                                        */
  size_t hbm_budget_bytes;    /* admission limit on the sum, over admitted requests, of the
                                 bytes of X, of the cores and of the slot workspace       */
  size_t arena_bytes;         /* slot workspace allocated at creation (<= the budget)       */
  int max_slots;              /* concurrent requests, 1..4096                               */
  int max_modes;              /* limits every request must meet: N <= max_modes,           */
  int64_t max_dim;            /*   every I_k <= max_dim,                                    */
  int max_rank;               /*   every rank <= max_rank (<= 16),                          */
  int64_t max_samples;        /*   J <= max_samples                                         */
  int max_sweeps;             /* default sweep cap, 1..TR_MAX_SERVED_SWEEPS                */
  double fit_tol;             /* default stop tolerance on |fit_s - fit_{s-1}|              */
  tr_dtype X_dtype;           /* dtype of every request's X                                 */
  tr_precision prec;          /* arithmetic of every request                                */
} tr_server_config;

/* One decomposition request. X and cores are DEVICE buffers owned by the caller; they must
 * stay valid (X unchanged) until the request is reported done. */
typedef struct tr_request {
  const void* X;                   /* device, row-major [dims[0]]...[dims[N-1]], X_dtype   */
  int N;
  int64_t dims[TR_MAX_MODES];
  int ranks[TR_MAX_MODES];
  int64_t J;                       /* samples per least-squares problem                     */
  uint64_t seed;                   /* Philox key of the request's draws (and its init)      */
  double* cores[TR_MAX_MODES];     /* device FP64 slice-major, receive the result           */
  int init_given;                  /* nonzero: cores[1..N-1] hold the initial cores         */
  int max_sweeps;                  /* 0 = the server's default                               */
  double fit_tol;                  /* < 0 = the server's default                             */
} tr_request;

typedef struct tr_result {
  int done;                        /* 0 while queued or running                             */
  tr_status status;                /* TR_OK (converged), TR_ERR_NOT_CONVERGED (sweep cap),
                                      TR_ERR_SINGULAR (non-finite fit), TR_ERR_CUDA          */
  int sweeps;                      /* completed sweeps                                       */
  int singular_updates;            /* updates whose normal matrix was singular (core kept)  */
  double fit;                      /* relative fit after the last sweep                      */
  double fit_change;               /* |fit - previous sweep's fit|                           */
  int64_t t_submit_ns;             /* CLOCK_MONOTONIC timestamps of submission, admission  */
  int64_t t_admit_ns;              /*   and of the end of the tick that finished it         */
  int64_t t_done_ns;
  double fit_history[TR_MAX_SERVED_SWEEPS];  /* fit after each sweep                      */
} tr_result;

typedef struct tr_server_stats {
  int64_t ticks;                   /* graph replays so far                                   */
  int64_t tick_ns;                 /* host time spent in ticks (admission + replay + wait)   */
  int64_t submitted, completed, rejected;
  int64_t updates;                 /* core updates performed                                  */
  int active;                      /* requests in slots                                      */
  int queued;                      /* requests waiting for admission                         */
  int peak_active;
  size_t charged_bytes;            /* current sum of admitted requests' charges              */
  size_t peak_charged_bytes;
} tr_server_stats;

/* Creates a server: checks the configuration, allocates the arena and the slot tables,
 * and captures one CUDA graph per slot-count bucket (8, 16, ... up to max_slots). */
tr_status tr_server_create(const tr_server_config* cfg, tr_server** out);
/* Stops the worker (if started), waits for the device and frees everything; requests still
 * queued or running are abandoned. */
void tr_server_destroy(tr_server* srv);
/* Message of the last failure of a call on this server (srv == NULL: of tr_server_create). */
const char* tr_server_last_error(const tr_server* srv);

/* Queues a request; thread-safe. Returns TR_ERR_INVALID_ARG for a request outside the
 * server's limits and TR_ERR_BUDGET for one whose charge alone exceeds the budget or the
 * arena; neither is queued. *ticket identifies the request in poll / wait. */
tr_status tr_server_submit(tr_server* srv, const tr_request* req, int64_t* ticket);

/* Runs one tick on the calling thread (not allowed while the worker runs): admits what
 * fits, replays the graph of the occupied slots, waits for it and retires finished
 * requests. *active (may be NULL) receives the number of occupied slots after the tick. */
tr_status tr_server_tick(tr_server* srv, int* active);

/* Starts / stops a native worker thread that ticks whenever requests are queued or running
 * and sleeps otherwise. */
tr_status tr_server_start(tr_server* srv);
tr_status tr_server_stop(tr_server* srv);

/* Result of a request, thread-safe. poll returns at once (out->done = 0 while the request
 * is queued or running); wait blocks until it is done or timeout_ms passes
 * (TR_ERR_TIMEOUT), ticking on the calling thread when no worker runs. A result can be read
 * any number of times until tr_server_release(ticket). Unknown tickets: TR_ERR_INVALID_ARG. */
tr_status tr_server_poll(tr_server* srv, int64_t ticket, tr_result* out);
tr_status tr_server_wait(tr_server* srv, int64_t ticket, int64_t timeout_ms, tr_result* out);
tr_status tr_server_release(tr_server* srv, int64_t ticket);
tr_status tr_server_get_stats(tr_server* srv, tr_server_stats* out);

/* Per-kernel timing. Between tr_profile_begin and tr_profile_end every kernel the context
 * launches is bracketed by a pair of CUDA events recorded on the launching stream.
 * tr_profile_end waits for `stream` and folds the event pairs into per-kernel totals
 * (milliseconds and launch counts) that tr_profile_entry reads by index
 * (0 <= i < tr_profile_count). tr_profile_begin clears earlier totals. */
tr_status tr_profile_begin(tr_ctx* ctx);
tr_status tr_profile_end(tr_ctx* ctx, tr_stream stream);
int tr_profile_count(const tr_ctx* ctx);
tr_status tr_profile_entry(const tr_ctx* ctx, int i, const char** name, double* total_ms,
                           int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* TRALS_H */
