// C ABI of libtrals.so: argument checks, workspace, and the Alg. 2 driver. Every step of
// the hot path runs in the kernels of this library; this file only validates, carves the
// workspace and issues launches on the caller's stream.
#include <cmath>
#include <cstdarg>
#include <map>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "batched.cuh"
#include "common.cuh"
#include "host_util.h"

struct tr_ctx {
  int device = 0;
  size_t budget = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  char* host_stage = nullptr;      // device buffers of tr_als_sampled_host
  size_t host_stage_bytes = 0;
  unsigned* d_err = nullptr;
  std::string last_error;
  // per-kernel profiler
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<const char*, size_t>> prof_marks;  // (kernel, first event index)
  std::map<std::string, std::pair<double, int64_t>> prof_tot;
  std::vector<std::pair<std::string, std::pair<double, int64_t>>> prof_snapshot;
  // CUDA graph of the last tr_als_sampled signature
  cudaStream_t cap = nullptr;       // internal stream, used only for capture
  cudaStream_t side = nullptr;      // second branch of each core update
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_info = nullptr;
  uint64_t* d_seed = nullptr;       // Philox key read by the captured kernels
  bool capturing = false;
  struct Mark { const char* name; cudaEvent_t a, b; };
  std::vector<Mark> graph_marks;    // profiler events captured into the graph
  cudaGraphExec_t gexec = nullptr;
  std::vector<uint64_t> gkey;
  bool gprof = false;
  // CUDA graph of the last batched launch geometry
  cudaGraphExec_t bexec = nullptr;
  std::vector<uint64_t> bkey;
  std::vector<trk::BInst> btab;     // host copy of the instance table
  tr_batched_tiles tiles{4, 64};    // launch shapes of the batched kernels
  tr_sampling sampling = TR_SAMPLING_LEVERAGE;   // draws of tr_als_sampled / batched
  tr_ls_rank ls_rank = TR_LS_RANK_STOP;          // rule for small pivots of the LS step
  long long wait_limit = -1;                     // polls per bounded wait (< 0: default)
  tr_factorization factorization = TR_FACTOR_DEFAULT;  // mixed path's factorisations
  int merge = 0;                                 // merge repeated draws in the drivers
};

namespace {

using namespace trk;

tr_status fail(tr_ctx* ctx, tr_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return s;
}

#define TR_CUDA(expr)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, TR_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));   \
  } while (0)

#define TR_TRY(expr)                       \
  do {                                     \
    tr_status s_ = (expr);                 \
    if (s_ != TR_OK) return s_;            \
  } while (0)

tr_status ensure_ws(tr_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->arena_bytes) return TR_OK;
  size_t want = bytes + bytes / 4;
  want = (want + (2u << 20) - 1) & ~size_t((2u << 20) - 1);
  if (ctx->budget && want + ctx->host_stage_bytes > ctx->budget) {
    want = bytes;
    if (want + ctx->host_stage_bytes > ctx->budget)
      return fail(ctx, TR_ERR_BUDGET, "workspace of %zu bytes exceeds the HBM budget of %zu",
                  bytes, ctx->budget);
  }
  // The old arena may still be read by queued work on any stream of this context.
  TR_CUDA(cudaDeviceSynchronize());
  if (ctx->arena) cudaFree(ctx->arena);
  ctx->arena = nullptr;
  ctx->arena_bytes = 0;
  if (cudaMalloc(&ctx->arena, want) != cudaSuccess) {
    cudaGetLastError();
    ctx->arena = nullptr;
    return fail(ctx, TR_ERR_OOM, "cudaMalloc of %zu workspace bytes failed", want);
  }
  ctx->arena_bytes = want;
  return TR_OK;
}

cudaStream_t S(tr_stream s) { return static_cast<cudaStream_t>(s); }

// Records an event pair around one launch when profiling is on. While a graph is being
// captured the events become nodes of that graph and belong to it.
struct Prof {
  tr_ctx* ctx;
  const char* name;
  cudaStream_t st;
  size_t first = 0;
  cudaEvent_t ga = nullptr, gb = nullptr;
  bool on;
  Prof(tr_ctx* c, const char* n, cudaStream_t s) : ctx(c), name(n), st(s), on(c->prof) {
    if (!on) return;
    if (ctx->capturing) {
      if (cudaEventCreate(&ga) != cudaSuccess || cudaEventCreate(&gb) != cudaSuccess) {
        on = false;
        return;
      }
      cudaEventRecordWithFlags(ga, st, cudaEventRecordExternal);  // a node of the graph
      return;
    }
    if (ctx->ev_used + 2 > ctx->ev_pool.size()) {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
        ctx->ev_pool.push_back(e);
      }
    }
    first = ctx->ev_used;
    ctx->ev_used += 2;
    cudaEventRecord(ctx->ev_pool[first], st);
  }
  ~Prof() {
    if (!on) return;
    if (ctx->capturing) {
      cudaEventRecordWithFlags(gb, st, cudaEventRecordExternal);
      ctx->graph_marks.push_back({name, ga, gb});
      return;
    }
    cudaEventRecord(ctx->ev_pool[first + 1], st);
    ctx->prof_marks.emplace_back(name, first);
  }
};

void add_prof(tr_ctx* ctx, const char* name, float ms) {
  auto& t = ctx->prof_tot[name];
  t.first += ms;
  t.second += 1;
}

void drop_graph(tr_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  for (auto& m : ctx->graph_marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  ctx->graph_marks.clear();
  ctx->gkey.clear();
}

#define TR_LAUNCH(name, expr)                     \
  do {                                            \
    Prof prof_(ctx, name, st);                    \
    TR_CUDA(expr);                                \
  } while (0)

// ------------------------------------------------------------------------------------
// Row a1: leverage-score distribution of one core.
// ------------------------------------------------------------------------------------
constexpr int kGramTiles = 64;   // Gram tile counters of launch_gram_dd (n <= 128: 10 tiles)

struct LevPass {  // one Cholesky-QR pass over an m x n row-major matrix (n = Gram size)
  double* partial; double* G; double* Lrow; double* Lcol; double* invdiag; int* keep; int* info;
  double* img;     // padded FP64 image of the factor for the row solves
  int splits;
  LevPrecond pre;  // the mixed drivers' preconditioned form (tall passes only)
};

LevPass carve_pass(Carver& c, int64_t rows, int cols, bool trans) {
  LevPass p{};
  const int n = trans ? static_cast<int>(rows) : cols;
  gram_workspace(rows, cols, trans, &p.splits);
  p.partial = c.take<double>(static_cast<size_t>(p.splits) * n * n);
  p.G = c.take<double>(static_cast<size_t>(n) * n);
  p.Lrow = c.take<double>(static_cast<size_t>(n) * n);
  p.Lcol = c.take<double>(static_cast<size_t>(n) * n);
  p.invdiag = c.take<double>(n);
  p.keep = c.take<int>(n);
  p.info = c.take<int>(1);
  p.img = reinterpret_cast<double*>(c.take<char>(trsm_image_bytes(n, false)));
  if (!trans && lev_precond_fits(rows, cols)) {
    p.pre.Ximg = reinterpret_cast<float*>(c.take<char>(trsm_image_bytes(n, true)));
    const size_t ld4 = static_cast<size_t>((n + 3) & ~3);
    p.pre.Uh = c.take<float>(n * ld4);
    p.pre.Ul = c.take<float>(n * ld4);
    p.pre.E = c.take<float>(n * ld4);
    p.pre.esq = c.take<float>(lev_precond_ctas(n));
    p.pre.state = c.take<int>(1);
    p.pre.lda_k = (n + 3) & ~3;
    p.pre.K_hi = reinterpret_cast<const float*>(p.Lrow);
    p.pre.K_lo = reinterpret_cast<const float*>(p.Lcol);
    p.pre.gph = c.take<float>(gram_dd_partial_floats(rows, cols));
    p.pre.gpl = c.take<float>(gram_dd_partial_floats(rows, cols));
  }
  return p;
}

// `mixed` (a single tall pass of the mixed-precision drivers): the double-float factorisation
// with FP64 fallback.
tr_status run_pass(tr_ctx* ctx, const LevPass& p, const double* A, int64_t rows, int cols,
                   int64_t lda, bool trans, double tol_scale, cudaStream_t st,
                   bool mixed = false, const float* A_hi = nullptr,
                   const float* A_lo = nullptr) {
  const int n = trans ? static_cast<int>(rows) : cols;
  if (mixed && !trans && A_hi) {
    // the mixed drivers' tall Gram in double-float from A's planes (written by the reduction)
    TR_LAUNCH("gram_f64", launch_gram_ff(A_hi, A_lo, rows, cols, lda, p.partial, p.splits, st));
  } else {
    TR_LAUNCH("gram_f64", launch_gram(A, rows, cols, lda, trans, p.partial, p.splits, st));
  }
  // the mixed tall pass: the reduction also writes the double-float planes of the Gram in
  // the factorisation's work-array layout (into Lrow / Lcol, free until the factor's tail)
  ReduceSplit sp;
  const bool presplit = mixed && n >= 4 && n <= 160;
  if (presplit) {
    sp.hi = reinterpret_cast<float*>(p.Lrow);
    sp.lo = reinterpret_cast<float*>(p.Lcol);
    sp.lda = (n + 3) & ~3;
  }
  TR_LAUNCH("reduce_gram", launch_reduce(p.partial, false, p.splits, static_cast<int64_t>(n) * n,
                                         n, n, n, n, p.G, n, nullptr, 0, st, sp));
  if (mixed) {
    const double eps = 2.220446049250313e-16, eps_ff = 9.094947017729282e-13;   // 2^-40
    TR_LAUNCH("cholesky_leverage",
              launch_cholesky_lev_mixed(p.G, n, tol_scale, tol_scale / eps * eps_ff, p.Lrow,
                                        p.Lcol, p.invdiag, p.keep, p.info, ctx->d_err, st,
                                        p.img, presplit ? sp.hi : nullptr,
                                        presplit ? sp.lo : nullptr));
    TR_LAUNCH("ff_image", launch_ff_image(p.Lrow, p.Lcol, n, p.info, p.img, st));
    return TR_OK;
  }
  TR_LAUNCH("cholesky_leverage", launch_cholesky(p.G, n, 1, tol_scale, p.Lrow, p.Lcol,
                                                   p.invdiag, p.keep, p.info, ctx->d_err, st,
                                                   p.img));
  return TR_OK;
}

size_t leverage_plan(Carver& c, int64_t I, int L, LevPass* p1, LevPass* p2, double** ell) {
  if (I >= L) {
    *p1 = carve_pass(c, I, L, false);
  } else {
    *p1 = carve_pass(c, I, L, true);                // K = A A^T (I x I) -> factor C
    *p2 = carve_pass(c, I, static_cast<int>(I), false);  // Gram of C (I x I)
  }
  *ell = c.take<double>(I);
  c.take<unsigned>(1 + kGramTiles);   // completion counters: the CDF step, then the Gram tiles
  return c.off;
}

size_t leverage_bytes(int64_t I, int L) {
  Carver c(nullptr);
  LevPass a, b;
  double* e;
  return leverage_plan(c, I, L, &a, &b, &e);
}

// Largest ||E||_F of the preconditioned series (TRALS_LEV_TAU, default 1e-2; 0 sends every
// distribution to the factorisation fallback, which the tests use to run it in a graph).
float lev_tau() {
  const char* e = getenv("TRALS_LEV_TAU");
  if (!e || !*e) return 1e-2f;
  const float v = strtof(e, nullptr);
  return v >= 0.f && v <= 1e-2f ? v : 1e-2f;
}

// The preconditioned form of the mixed drivers' tall leverage scores (on unless
// TRALS_LEV_PRECOND=0, which keeps the double-float factorisation for every update).
bool precond_enabled() {
  const char* e = getenv("TRALS_LEV_PRECOND");
  return !(e && e[0] == '0');
}

// Leverage scores of the rows of the I x L row-major matrix `mat` (a core's G_(2), or any
// matrix with the same column space) and, from them, p and the CDF (unless *skip != 0).
// `mixed` (the mixed-precision drivers): a tall matrix's Gram is factored in double-float
// when no pivot is small (about 46 significant bits; rank decisions stay FP64).
tr_status leverage_dist(tr_ctx* ctx, char* ws, const double* mat, int64_t I, int L, double* p,
                        double* cdf, const int* skip, cudaStream_t st,
                        cudaEvent_t wait_before_rows = nullptr, bool mixed = false,
                        const float* mat_hi = nullptr, const float* mat_lo = nullptr) {
  Carver c(ws);
  LevPass p1{}, p2{};
  double* ell;
  leverage_plan(c, I, L, &p1, &p2, &ell);
  if (I < L && leverage_jacobi_fits(I, L)) {
    // Wide G_(2) with few rows: one-sided Jacobi in one CTA, the singular-value rank rule
    if (wait_before_rows) TR_CUDA(cudaStreamWaitEvent(st, wait_before_rows, 0));
    TR_LAUNCH("leverage_jacobi", launch_leverage_jacobi(mat, I, L, L, ell, p, cdf, skip,
                                                        ctx->d_err, st));
    return TR_OK;
  }
  unsigned* counter = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(ell) +
                                                  ((I * sizeof(double) + 255) & ~size_t(255)));
  const double eps = 2.220446049250313e-16;
  const double tol = static_cast<double>(I > L ? I : L) * eps;
  TR_CUDA(cudaMemsetAsync(counter, 0, (1 + kGramTiles) * sizeof(unsigned), st));
  const CdfEpilogue ep{counter, p, cdf, skip, ctx->d_err};
  if (I >= L && mixed && mat_hi && p1.pre.state && precond_enabled()) {
    // FP32 preconditioner and a short series (lev_precond.cu); the double-float
    // factorisation, its image and the FP64 row solves run only when its device flag says so
    const int n = L;
    ReduceSplit sp;
    sp.hi = reinterpret_cast<float*>(p1.Lrow);
    sp.lo = reinterpret_cast<float*>(p1.Lcol);
    sp.lda = (n + 3) & ~3;
    TR_LAUNCH("gram_dd", launch_gram_dd(mat_hi, mat_lo, I, n, n, p1.pre.gph, p1.pre.gpl,
                                        counter + 1, sp.hi, sp.lo, sp.lda, p1.G, st));
    TR_LAUNCH("lev_factor", launch_lev_precond(0, p1.pre, n, I, mat_hi, mat_lo, L, ell, ep, st));
    TR_LAUNCH("lev_u", launch_lev_precond(1, p1.pre, n, I, mat_hi, mat_lo, L, ell, ep, st));
    TR_LAUNCH("lev_e", launch_lev_precond(2, p1.pre, n, I, mat_hi, mat_lo, L, ell, ep, st));
    if (wait_before_rows) TR_CUDA(cudaStreamWaitEvent(st, wait_before_rows, 0));
    LevPrecond lp = p1.pre;
    lp.tau = lev_tau();
    TR_LAUNCH("lev_rows", launch_lev_precond(3, lp, n, I, mat_hi, mat_lo, L, ell, ep, st));
    // the fallback: issued always, each launch exits at once unless the device flag asks for
    // it (a conditional graph node measured slower than these three launches)
    const int* gate = p1.pre.state;
    const double eps_ff = 9.094947017729282e-13;   // 2^-40
    TR_LAUNCH("cholesky_leverage",
              launch_cholesky_lev_mixed(p1.G, n, tol, tol / eps * eps_ff, p1.Lrow, p1.Lcol,
                                        p1.invdiag, p1.keep, p1.info, ctx->d_err, st, p1.img,
                                        sp.hi, sp.lo, gate));
    TR_LAUNCH("ff_image", launch_ff_image(p1.Lrow, p1.Lcol, n, p1.info, p1.img, st, gate));
    CdfEpilogue ep2 = ep;
    ep2.run_if = gate;
    TR_LAUNCH("leverage_rows", launch_trsm(0, false, L, p1.Lrow, p1.Lcol, p1.invdiag, nullptr, I,
                                           mat, L, nullptr, 1, 1, nullptr, ell, st, p1.img,
                                           nullptr, &ep2));
  } else if (I >= L) {
    TR_TRY(run_pass(ctx, p1, mat, I, L, L, false, tol, st, mixed, mat_hi, mat_lo));
    if (wait_before_rows) TR_CUDA(cudaStreamWaitEvent(st, wait_before_rows, 0));
    TR_LAUNCH("leverage_rows", launch_trsm(0, false, L, p1.Lrow, p1.Lcol, p1.invdiag, nullptr, I,
                                           mat, L, nullptr, 1, 1, nullptr, ell, st, p1.img,
                                           nullptr, &ep));
  } else {
    // Wide G_(2): the range of A is that of C with A A^T = C C^T; ell(A) = ell(C).
    const int n = static_cast<int>(I);
    TR_TRY(run_pass(ctx, p1, mat, I, L, L, true, tol, st));
    TR_TRY(run_pass(ctx, p2, p1.Lrow, I, n, n, false, tol, st));
    if (wait_before_rows) TR_CUDA(cudaStreamWaitEvent(st, wait_before_rows, 0));
    TR_LAUNCH("leverage_rows", launch_trsm(0, false, n, p2.Lrow, p2.Lcol, p2.invdiag, nullptr, I,
                                           p1.Lrow, n, nullptr, 1, 1, nullptr, ell, st, p2.img,
                                           nullptr, &ep));
  }
  return TR_OK;
}

tr_status leverage_run(tr_ctx* ctx, char* ws, const double* core, int64_t I, int Rl, int Rr,
                       double* p, double* cdf, cudaStream_t st, bool mixed = false) {
  return leverage_dist(ctx, ws, core, I, Rl * Rr, p, cdf, nullptr, st, nullptr, mixed);
}

// ------------------------------------------------------------------------------------
// Rows a5 + a6: normal equations, Cholesky, solve, refinement.
// ------------------------------------------------------------------------------------
struct SolvePlan {
  void* partial; double* M; double* BT; double* Lrow; double* Lcol; double* invdiag;
  int* keep; int* info; void* limg; float* mimg; float* wimg; int splits;
  float* bt_hi = nullptr; float* bt_lo = nullptr;   // double-float planes of B^T (mixed)
  int* fast = nullptr;   // the one-CTA FP32 factor-and-inverse succeeded (mixed, L <= 128)
};

bool use_tensor_cores(bool f64) {
  if (f64) return false;
  const char* e = getenv("TRALS_SIMT_CONTRACT");
  return !(e && e[0] == '1');
}

size_t solve_plan(Carver& c, int64_t J, int L, int64_t I, bool f64, SolvePlan* s) {
  const size_t pbytes = use_tensor_cores(f64) ? normal_eq_tc_workspace(J, L, I, &s->splits)
                                              : normal_eq_workspace(J, L, I, f64, &s->splits);
  s->partial = c.take<char>(pbytes);
  s->M = c.take<double>(static_cast<size_t>(L) * L);
  s->BT = c.take<double>(static_cast<size_t>(I) * L);
  s->Lrow = c.take<double>(static_cast<size_t>(L) * L);
  s->Lcol = c.take<double>(static_cast<size_t>(L) * L);
  s->invdiag = c.take<double>(L);
  s->keep = c.take<int>(L);
  s->info = c.take<int>(1);
  s->limg = c.take<char>(trsm_image_bytes(L, !f64));
  s->mimg = f64 ? nullptr : reinterpret_cast<float*>(c.take<char>(trsm_image_bytes(L, true)));
  s->wimg = f64 ? nullptr : reinterpret_cast<float*>(c.take<char>(trsm_image_bytes(L, true)));
  s->bt_hi = f64 ? nullptr : c.take<float>(static_cast<size_t>(I) * L);
  s->bt_lo = f64 ? nullptr : c.take<float>(static_cast<size_t>(I) * L);
  s->fast = f64 ? nullptr : c.take<int>(1);
  return c.off;
}

size_t solve_bytes(int64_t J, int L, int64_t I, bool f64) {
  Carver c(nullptr);
  SolvePlan s;
  return solve_plan(c, J, L, I, f64, &s);
}

tr_status solve_contract(tr_ctx* ctx, const SolvePlan& s, const void* A, const void* Y,
                         bool f64, int64_t J, int L, int64_t I, cudaStream_t st,
                         const int64_t* jdev = nullptr, bool bt_planes = false) {
  const int64_t ld = L + I;
  if (use_tensor_cores(f64)) {
    TR_LAUNCH("normal_eq_tc", launch_normal_eq_tc(static_cast<const float*>(A),
                                                  static_cast<const float*>(Y), J, L, I,
                                                  static_cast<float*>(s.partial), s.splits,
                                                  ctx->d_err, st, ctx->wait_limit, jdev));
  } else {
    TR_LAUNCH("normal_eq", launch_normal_eq(A, Y, f64, J, L, I, s.partial, s.splits, st, jdev));
  }
  // mixed: the reduction also writes M's FP32 values in the factorisation's work-array
  // layout (into Lrow, free until an FP64 fallback) and M's FP32 image
  ReduceSplit sp;
  if (!f64 && L >= 4 && L <= 160) {
    sp.hi = reinterpret_cast<float*>(s.Lrow);
    sp.lda = (L + 3) & ~3;
    sp.img = s.mimg;
    sp.np = L + 1;
  }
  if (bt_planes && s.bt_hi) {
    sp.t_hi = s.bt_hi;
    sp.t_lo = s.bt_lo;
  }
  TR_LAUNCH("reduce_MB", launch_reduce(s.partial, !f64, s.splits, L * ld, ld, L, ld, L, s.M, L,
                                       s.BT, L, st, sp));
  return TR_OK;
}

// The flag of the mixed LS step's one-CTA FP32 factor-and-inverse (launch_cholesky_mixed),
// or nullptr where that form does not apply (FP64 arithmetic or factorisations, L > 128).
int* tiles_flag(const tr_ctx* ctx, const SolvePlan& s, bool f64, int L) {
  return (!f64 && ctx->factorization != TR_FACTOR_FP64 && L >= 4 && L <= 128) ? s.fast : nullptr;
}

tr_status solve_cholesky(tr_ctx* ctx, const SolvePlan& s, bool f64, int L, cudaStream_t st) {
  const double eps = 2.220446049250313e-16;
  const int mode = ctx->ls_rank == TR_LS_RANK_DROP ? 1 : 0;
  if (!f64 && ctx->factorization == TR_FACTOR_FP64) {
    // FP64 factorisation, FP32 image of the factor for the FP32 solves with refinement
    TR_LAUNCH("cholesky_solve",
              launch_cholesky(s.M, L, mode, static_cast<double>(L) * eps, s.Lrow, s.Lcol,
                              s.invdiag, s.keep, s.info, ctx->d_err, st, nullptr,
                              static_cast<float*>(s.limg), s.mimg));
    return TR_OK;
  }
  if (!f64) {
    const double eps32 = 1.1920928955078125e-07;
    TR_LAUNCH("cholesky_solve",
              launch_cholesky_mixed(s.M, L, mode, static_cast<double>(L) * eps,
                                    static_cast<double>(L) * eps32, s.Lrow, s.Lcol, s.invdiag,
                                    s.keep, s.info, ctx->d_err, st, static_cast<float*>(s.limg),
                                    s.mimg,
                                    L >= 4 && L <= 160 ? reinterpret_cast<float*>(s.Lrow)
                                                       : nullptr,
                                    s.wimg, tiles_flag(ctx, s, f64, L)));
    return TR_OK;
  }
  TR_LAUNCH("cholesky_solve",
            launch_cholesky(s.M, L, mode, static_cast<double>(L) * eps, s.Lrow, s.Lcol, s.invdiag,
                            s.keep, s.info, ctx->d_err, st, static_cast<double*>(s.limg),
                            nullptr, nullptr));
  return TR_OK;
}

tr_status solve_rhs(tr_ctx* ctx, const SolvePlan& s, int Rl, int Rr, int64_t I, bool refine,
                    double* core_out, cudaStream_t st) {
  const int L = Rl * Rr;
  if (refine && solve_inv_fits(L)) {
    TR_LAUNCH("solve_rhs", launch_solve_inv(L, static_cast<const float*>(s.limg), s.mimg,
                                            s.invdiag, s.info, I, s.BT, L, Rl, Rr, core_out,
                                            s.wimg, st, tiles_flag(ctx, s, !refine, L)));
    return TR_OK;
  }
  TR_LAUNCH("solve_rhs", launch_trsm(refine ? 2 : 1, refine, L, s.Lrow, s.Lcol, s.invdiag, s.info,
                                      I, s.BT, L, s.M, Rl, Rr, core_out, nullptr, st, s.limg,
                                      s.mimg));
  return TR_OK;
}

tr_status solve_factor(tr_ctx* ctx, const SolvePlan& s, bool f64, int Rl, int Rr, int64_t I,
                       bool refine, double* core_out, cudaStream_t st) {
  TR_TRY(solve_cholesky(ctx, s, f64, Rl * Rr, st));
  return solve_rhs(ctx, s, Rl, Rr, I, refine, core_out, st);
}

tr_status solve_run(tr_ctx* ctx, char* ws, const void* A, const void* Y, bool f64, int64_t J,
                    int Rl, int Rr, int64_t I, bool refine, double* core_out, cudaStream_t st) {
  const int L = Rl * Rr;
  Carver c(ws);
  SolvePlan s;
  solve_plan(c, J, L, I, f64, &s);
  TR_TRY(solve_contract(ctx, s, A, Y, f64, J, L, I, st));
  return solve_factor(ctx, s, f64, Rl, Rr, I, refine, core_out, st);
}

// One core update's LS step and distribution update as two concurrent branches. Since
// M = A~^T A~ is nonsingular whenever the solve succeeds, the new core's G_(2) = Z^T =
// B^T M^-1 has the column space of B^T, so p^(n) is computed from B^T on the side stream
// while the main stream factors M and solves. The CDF step joins both and keeps the old
// distribution if the solve reported a singular system (the core is then unchanged).
tr_status update_run(tr_ctx* ctx, char* ws, size_t solve_ws, const void* A, const void* Y,
                     bool f64, int64_t J, int Rl, int Rr, int64_t I, double* core_out, double* p,
                     double* cdf, cudaStream_t st, cudaStream_t side,
                     const int64_t* jdev = nullptr) {
  const int L = Rl * Rr;
  Carver c(ws);
  SolvePlan s;
  solve_plan(c, J, L, I, f64, &s);
  const bool mixed_lev = !f64 && ctx->factorization != TR_FACTOR_FP64;
  // the distribution branch's tall Gram of B^T runs in double-float from B^T's planes
  const bool bt_planes = p && mixed_lev && ctx->ls_rank != TR_LS_RANK_DROP && I >= L;
  TR_TRY(solve_contract(ctx, s, A, Y, f64, J, L, I, st, jdev, bt_planes));
  if (!p) {   // uniform sampling: the new core needs no distribution
    TR_TRY(solve_cholesky(ctx, s, f64, L, st));
    return solve_rhs(ctx, s, Rl, Rr, I, !f64, core_out, st);
  }
  if (ctx->ls_rank == TR_LS_RANK_DROP) {
    // A dropped column is only nearly dependent on the kept ones, and its unknowns are set to
    // zero: the new core's column space is that of the kept columns of B^T, not of B^T. The
    // distribution is therefore the leverage of the new core itself (Alg. 2, "update n-th
    // distribution"), formed after the solve. The core's slice-major rows are its G_(2) rows
    // with the columns permuted, which leaves the leverage scores unchanged.
    TR_TRY(solve_cholesky(ctx, s, f64, L, st));
    TR_TRY(solve_rhs(ctx, s, Rl, Rr, I, !f64, core_out, st));
    return leverage_dist(ctx, ws + solve_ws, core_out, I, L, p, cdf, s.info, st, nullptr,
                         mixed_lev);
  }
  TR_CUDA(cudaEventRecord(ctx->ev_fork, st));
  TR_CUDA(cudaStreamWaitEvent(side, ctx->ev_fork, 0));
  TR_TRY(solve_cholesky(ctx, s, f64, L, st));
  // The side branch needs the solve's Cholesky status (info) only in its last kernel, to
  // keep the old distribution when the core was not updated.
  TR_CUDA(cudaEventRecord(ctx->ev_info, st));
  TR_TRY(solve_rhs(ctx, s, Rl, Rr, I, !f64, core_out, st));
  TR_TRY(leverage_dist(ctx, ws + solve_ws, s.BT, I, L, p, cdf, s.info, side, ctx->ev_info,
                       mixed_lev, bt_planes ? s.bt_hi : nullptr,
                       bt_planes ? s.bt_lo : nullptr));
  TR_CUDA(cudaEventRecord(ctx->ev_join, side));
  TR_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  return TR_OK;
}

// ------------------------------------------------------------------------------------
// Validation helpers.
// ------------------------------------------------------------------------------------
tr_status check_ctx(tr_ctx* ctx) {
  return ctx ? TR_OK : TR_ERR_INVALID_ARG;
}

tr_status check_shape(tr_ctx* ctx, int N, const int64_t* dims, const int* ranks) {
  if (N < 2 || N > kMaxModes) return fail(ctx, TR_ERR_INVALID_ARG, "N=%d outside [2, %d]", N, kMaxModes);
  if (!dims) return fail(ctx, TR_ERR_INVALID_ARG, "dims is NULL");
  for (int k = 0; k < N; ++k)
    if (dims[k] < 1 || dims[k] > INT32_MAX)
      return fail(ctx, TR_ERR_INVALID_ARG, "dims[%d]=%lld outside [1, 2^31-1]", k,
                  static_cast<long long>(dims[k]));
  if (ranks) {
    for (int k = 0; k < N; ++k)
      if (ranks[k] < 1 || ranks[k] > 16)
        return fail(ctx, TR_ERR_INVALID_ARG, "ranks[%d]=%d outside [1, 16]", k, ranks[k]);
  }
  return TR_OK;
}

int rl_of(const int* ranks, int N, int k) { return ranks[(k - 1 + N) % N]; }

tr_status read_device_error(tr_ctx* ctx, cudaStream_t st) {
  unsigned h = 0;
  TR_CUDA(cudaStreamSynchronize(st));
  TR_CUDA(cudaMemcpy(&h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost));
  TR_CUDA(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
  if (h & kErrTimeout) return fail(ctx, TR_ERR_TIMEOUT, "a bounded device wait expired");
  if (h & kErrBadIndex) return fail(ctx, TR_ERR_INVALID_ARG, "a sample index was out of range");
  if (h & kErrSingular)
    return fail(ctx, TR_ERR_SINGULAR, "non-positive pivot in the normal equations or a zero core");
  return TR_OK;
}

// The Alg. 2 driver on device buffers: plan the workspace (outside any capture), then issue
// every launch of one call on a stream.
struct AlsPlan {
  const void* X; tr_dtype xdt; int N; const int64_t* dims; const int* ranks; int64_t J;
  int sweeps; tr_precision prec; const double* const* init; double* const* cores;
  const int64_t* Js = nullptr;   // per-sweep sample sizes (Sec. 4.2), or null: J for all;
                                 // J is then their maximum (workspace)
  const int64_t* Jupd = nullptr; // per-update sample sizes [sweeps][N] (Sec. 4.2), or null
  std::vector<double*> p, cdf;
  int32_t* idx; double* w; void* A; void* Y; char* ws;
  int32_t* idx2 = nullptr; double* w2 = nullptr; int64_t* jm = nullptr;   // merged draws
  size_t solve_ws;   // bytes of the stage region used by the LS step; leverage follows it
  // per mode: a copy of X with that mode last (contiguous fibres), or null; and the element
  // strides of every mode in that copy
  void* Xm[kMaxModes] = {};
  int64_t mstride[kMaxModes][kMaxModes] = {};
  unsigned copy_mask = 0;
};

// A copy of X with mode n last is made for a strided mode when the decomposition's scattered
// fibre reads would move more DRAM bytes than the copy: each scattered element costs about
// 64 bytes (measured: ncu showed about 100 bytes of DRAM reads per 4-byte element of the
// strided modes of the 500^3 tensor), the copy 2 |X| (read and write). TRALS_PERMUTE=0 turns
// the copies off.
bool permute_enabled() {
  const char* e = getenv("TRALS_PERMUTE");
  return !(e && e[0] == '0');
}

unsigned choose_copies(const AlsPlan& P, size_t xbytes) {
  if (!permute_enabled()) return 0;
  int64_t stride[kMaxModes];
  row_major_strides(P.N, P.dims, stride);
  unsigned mask = 0;
  for (int n = 0; n < P.N; ++n) {
    if (stride[n] < 8) continue;
    const double scattered = static_cast<double>(P.sweeps) * static_cast<double>(P.J) *
                             static_cast<double>(P.dims[n]) * 64.0;
    if (scattered >= 2.0 * static_cast<double>(xbytes)) mask |= 1u << n;
  }
  return mask;
}

tr_status als_plan(tr_ctx* ctx, AlsPlan& P) {
  const int N = P.N;
  const bool f64 = P.prec == TR_PREC_FP64;
  const size_t es = f64 ? 8 : 4;
  int64_t Imax = 0, Isum = 0;
  int Lmax = 0;
  for (int k = 0; k < N; ++k) {
    Imax = P.dims[k] > Imax ? P.dims[k] : Imax;
    Isum += P.dims[k];
    const int L = rl_of(P.ranks, N, k) * P.ranks[k];
    Lmax = L > Lmax ? L : Lmax;
  }
  auto carve = [&](Carver& c, double** pb, double** cb) {
    *pb = c.take<double>(Isum);
    *cb = c.take<double>(Isum);
    P.idx = c.take<int32_t>(static_cast<size_t>(P.J) * (N - 1));
    P.w = c.take<double>(P.J);
    P.A = c.take<char>(static_cast<size_t>(P.J) * Lmax * es);
    P.Y = c.take<char>(static_cast<size_t>(P.J) * Imax * es);
    if (ctx->merge) {
      P.idx2 = c.take<int32_t>(static_cast<size_t>(P.J) * (N - 1));
      P.w2 = c.take<double>(P.J);
      P.jm = c.take<int64_t>(1);
    }
  };
  double *pb, *cb;
  Carver dry(nullptr);
  carve(dry, &pb, &cb);
  const size_t persist = (dry.off + 255) & ~size_t(255);
  size_t stage = 0, solve_max = 0;
  for (int k = 0; k < N; ++k) {
    const int L = rl_of(P.ranks, N, k) * P.ranks[k];
    const size_t b = (solve_bytes(P.J, L, P.dims[k], f64) + 255) & ~size_t(255);
    solve_max = b > solve_max ? b : solve_max;
  }
  for (int k = 0; k < N; ++k) {
    const int L = rl_of(P.ranks, N, k) * P.ranks[k];
    const size_t a = leverage_bytes(P.dims[k], L);
    stage = solve_max + a > stage ? solve_max + a : stage;
  }
  P.solve_ws = solve_max;
  // contiguous copies of X for strided modes, when they pay and memory allows
  int64_t numel = 1;
  for (int k = 0; k < N; ++k) numel *= P.dims[k];
  const size_t xbytes = (static_cast<size_t>(numel) * (P.xdt == TR_F64 ? 8 : 4) + 255) & ~size_t(255);
  P.copy_mask = choose_copies(P, xbytes);
  size_t ncopy = 0;
  for (int n = 0; n < N; ++n) ncopy += (P.copy_mask >> n) & 1u;
  if (ncopy) {
    const size_t need = persist + stage + ncopy * xbytes;
    size_t free_b = 0, total_b = 0;
    bool fits = need <= ctx->arena_bytes;
    if (!fits && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
      fits = need + need / 4 <= free_b + ctx->arena_bytes;
    cudaGetLastError();
    if (ctx->budget && need + ctx->host_stage_bytes > ctx->budget) fits = false;
    if (!fits) {
      P.copy_mask = 0;
      ncopy = 0;
    }
  }
  TR_TRY(ensure_ws(ctx, persist + ncopy * xbytes + stage));
  Carver c(ctx->arena);
  carve(c, &pb, &cb);
  char* copies = ctx->arena + persist;
  for (int n = 0; n < N; ++n) {
    P.Xm[n] = nullptr;
    if (!((P.copy_mask >> n) & 1u)) continue;
    P.Xm[n] = copies;
    copies += xbytes;
    // strides in the copy: the other modes in their order, then mode n
    int64_t run = P.dims[n];
    P.mstride[n][n] = 1;
    for (int k = N - 1; k >= 0; --k) {
      if (k == n) continue;
      P.mstride[n][k] = run;
      run *= P.dims[k];
    }
  }
  P.ws = ctx->arena + persist + ncopy * xbytes;
  P.p.resize(N);
  P.cdf.resize(N);
  int64_t off = 0;
  for (int k = 0; k < N; ++k) { P.p[k] = pb + off; P.cdf[k] = cb + off; off += P.dims[k]; }
  return TR_OK;
}

tr_status als_issue(tr_ctx* ctx, const AlsPlan& P, uint64_t seed, const uint64_t* seed_dev,
                    cudaStream_t st, cudaStream_t side) {
  const int N = P.N;
  const bool f64 = P.prec == TR_PREC_FP64;
  const int64_t* dims = P.dims;
  const int* ranks = P.ranks;
  for (int k = 1; k < N; ++k) {
    const size_t count = static_cast<size_t>(dims[k]) * rl_of(ranks, N, k) * ranks[k];
    if (P.init) {
      TR_CUDA(cudaMemcpyAsync(P.cores[k], P.init[k], count * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
    } else {
      TR_LAUNCH("init_normal", launch_init_normal(P.cores[k], static_cast<int64_t>(count), seed,
                                                  static_cast<uint32_t>(k), seed_dev, st));
    }
  }
  // contiguous copies of X for the strided modes (made every call: X may change)
  for (int n = 0; n < N; ++n) {
    if (!P.Xm[n]) continue;
    int64_t pre = 1, post = 1;
    for (int k = 0; k < n; ++k) pre *= dims[k];
    for (int k = n + 1; k < N; ++k) post *= dims[k];
    TR_LAUNCH("mode_last", launch_mode_last(P.X, P.xdt == TR_F64, pre, dims[n], post, P.Xm[n],
                                            st));
  }
  const bool uni = ctx->sampling == TR_SAMPLING_UNIFORM;
  if (!uni)
    for (int k = 1; k < N; ++k)
      TR_TRY(leverage_run(ctx, P.ws, P.cores[k], dims[k], rl_of(ranks, N, k), ranks[k], P.p[k],
                          P.cdf[k], st, !f64 && ctx->factorization != TR_FACTOR_FP64));
  int64_t stride[kMaxModes];
  row_major_strides(N, dims, stride);
  const bool x64 = P.xdt == TR_F64;
  for (int s = 0; s < P.sweeps; ++s) {
    for (int n = 0; n < N; ++n) {
      SampleArgs sa{};
      ChainArgs ca{};
      GatherArgs ga{};
      sa.npos = ca.npos = ga.npos = N - 1;
      sa.seed_dev = seed_dev;
      sa.uniform = uni ? 1 : 0;
      for (int m = 0; m < N - 1; ++m) {
        const int mode = (n + 1 + m) % N;
        sa.p[m] = P.p[mode];
        sa.cdf[m] = P.cdf[mode];
        sa.I[m] = ca.I[m] = ga.I[m] = dims[mode];
        ca.core[m] = P.cores[mode];
        ca.rl[m] = rl_of(ranks, N, mode);
        ca.rr[m] = ranks[mode];
        ga.stride[m] = stride[mode];
      }
      ga.In = dims[n];
      ga.stride_n = stride[n];
      const void* Xn = P.X;
      if (P.Xm[n]) {   // the copy with mode n last: contiguous fibres
        for (int m = 0; m < N - 1; ++m) ga.stride[m] = P.mstride[n][(n + 1 + m) % N];
        ga.stride_n = 1;
        Xn = P.Xm[n];
      }
      const uint64_t uid = static_cast<uint64_t>(s) * N + n;
      const int64_t Jn = P.Jupd ? P.Jupd[static_cast<int64_t>(s) * N + n]
                                : (P.Js ? P.Js[s] : P.J);
      MergeArgs ma{};
      const bool merge = ctx->merge && P.jm && merge_fits(Jn, N - 1, sa.I, &ma);
      if (merge) {
        // Sec. 4.2: draws, then one row per distinct multi-index with weight sqrt(count) w;
        // the rows, fibres and contraction take the merged count from device memory
        TR_LAUNCH("sample", launch_sample(sa, Jn, seed, uid, P.idx, P.w, st));
        TR_LAUNCH("merge", launch_merge(P.idx, P.w, Jn, N - 1, ma, P.idx2, P.w2, P.jm, st));
        SampleArgs sg = sa;
        sg.given_idx = P.idx2;
        sg.given_w = P.w2;
        sg.jdev = P.jm;
        TR_LAUNCH("sample_chain", launch_sample_chain(sg, ca, Jn, seed, uid, P.idx, P.w, P.A,
                                                      f64, st, &ga, Xn, x64, P.Y));
      } else {
        TR_LAUNCH("sample_chain", launch_sample_chain(sa, ca, Jn, seed, uid, P.idx, P.w, P.A,
                                                      f64, st, &ga, Xn, x64, P.Y));
      }
      const int Rl = rl_of(ranks, N, n), Rr = ranks[n];
      TR_TRY(update_run(ctx, P.ws, P.solve_ws, P.A, P.Y, f64, Jn, Rl, Rr, dims[n], P.cores[n],
                        uni ? nullptr : P.p[n], uni ? nullptr : P.cdf[n], st, side,
                        merge ? P.jm : nullptr));
    }
  }
  return TR_OK;
}

std::vector<uint64_t> als_key(const tr_ctx* ctx, const AlsPlan& P) {
  std::vector<uint64_t> k;
  auto u = [&](uint64_t v) { k.push_back(v); };
  u(reinterpret_cast<uintptr_t>(P.X));
  u(P.xdt);
  u(P.N);
  for (int i = 0; i < P.N; ++i) {
    u(static_cast<uint64_t>(P.dims[i]));
    u(static_cast<uint64_t>(P.ranks[i]));
    u(reinterpret_cast<uintptr_t>(P.cores[i]));
    u(P.init ? reinterpret_cast<uintptr_t>(P.init[i]) : 0);
  }
  u(static_cast<uint64_t>(P.J));
  if (P.Js)
    for (int s = 0; s < P.sweeps; ++s) u(static_cast<uint64_t>(P.Js[s]));
  u(P.Jupd ? 1 : 0);
  if (P.Jupd)
    for (int64_t e = 0; e < static_cast<int64_t>(P.sweeps) * P.N; ++e)
      u(static_cast<uint64_t>(P.Jupd[e]));
  u(static_cast<uint64_t>(ctx->merge));
  u(static_cast<uint64_t>(P.sweeps));
  u(P.prec);
  u(P.init ? 1 : 0);
  u(reinterpret_cast<uintptr_t>(ctx->arena));
  u(ctx->arena_bytes);
  u(static_cast<uint64_t>(ctx->sampling));
  u(static_cast<uint64_t>(ctx->ls_rank));
  u(static_cast<uint64_t>(ctx->wait_limit));
  u(static_cast<uint64_t>(ctx->factorization));
  u(precond_enabled() ? 1 : 0);
  {
    const float t = lev_tau();
    uint32_t b;
    memcpy(&b, &t, sizeof b);
    u(b);
  }
  u(P.copy_mask);
  return k;
}

bool graphs_enabled() {
  const char* e = getenv("TRALS_NO_GRAPH");
  return !(e && e[0] == '1');
}

// One whole call: plan, then either issue directly or (re)capture and launch the graph.
tr_status als_run(tr_ctx* ctx, AlsPlan& P, uint64_t seed, cudaStream_t st) {
  TR_TRY(als_plan(ctx, P));
  if (!graphs_enabled()) return als_issue(ctx, P, seed, nullptr, st, ctx->side);
  std::vector<uint64_t> key = als_key(ctx, P);
  if (!ctx->gexec || key != ctx->gkey || ctx->gprof != ctx->prof) {
    drop_graph(ctx);
    cudaGraph_t g = nullptr;
    ctx->capturing = true;
    TR_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    tr_status s = als_issue(ctx, P, 0, ctx->d_seed, ctx->cap, ctx->side);
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
    ctx->capturing = false;
    if (s != TR_OK) {
      if (g) cudaGraphDestroy(g);
      drop_graph(ctx);
      return s;
    }
    if (e != cudaSuccess) {
      drop_graph(ctx);
      return fail(ctx, TR_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ctx->gexec = nullptr;
      drop_graph(ctx);
      return fail(ctx, TR_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    ctx->gkey = key;
    ctx->gprof = ctx->prof;
  }
  TR_CUDA(cudaMemcpyAsync(ctx->d_seed, &seed, sizeof seed, cudaMemcpyHostToDevice, st));
  TR_CUDA(cudaGraphLaunch(ctx->gexec, st));
  return TR_OK;
}

// After a synchronised graph launch, fold its captured profiler events into the totals.
tr_status fold_graph_marks(tr_ctx* ctx) {
  if (!ctx->gexec || !ctx->gprof || !graphs_enabled()) return TR_OK;
  // Best effort: a timing that cannot be read is skipped, the call itself succeeded.
  for (const auto& m : ctx->graph_marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) add_prof(ctx, m.name, ms);
    else cudaGetLastError();
  }
  return TR_OK;
}

// ------------------------------------------------------------------------------------
// Batched driver.
// ------------------------------------------------------------------------------------
tr_status batched_issue(tr_ctx* ctx, const BLaunch& bl, int nmax_modes, int steps, bool draw,
                        cudaStream_t st) {
  if (draw) TR_CUDA(bl_init_cores(bl, st));
  if (bl.leverage)
    for (int k = 1; k < nmax_modes; ++k)
      TR_CUDA(issue_leverage(bl, 0, k, ctx->d_err, st, nullptr));
  const StepStreams ss{st, ctx->side, ctx->ev_fork, ctx->ev_info, ctx->ev_join};
  for (int step = 0; step < steps; ++step) TR_CUDA(issue_step(bl, step, ctx->d_err, ss));
  return TR_OK;
}

}  // namespace

// ======================================================================================
// Public entry points
// ======================================================================================
extern "C" {

static std::string g_create_error;  // message of the last failed tr_create / tr_solve_noalloc

tr_status tr_create(tr_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return TR_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) {
    g_create_error = std::string("no CUDA device ") + std::to_string(device) + ": " +
                     (e != cudaSuccess ? cudaGetErrorString(e) : "index out of range");
    cudaGetLastError();
    return TR_ERR_INVALID_ARG;
  }
  tr_ctx* ctx = new tr_ctx;
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  DeviceGuard g(device);
  const char* step = "cudaSetDevice";
  const char* which = "";
  e = g.ok ? cudaSuccess : cudaErrorInvalidDevice;
  if (e == cudaSuccess) { step = "cudaMalloc(status)"; e = cudaMalloc(&ctx->d_err, 256); }
  if (e == cudaSuccess) { step = "cudaMemset(status)"; e = cudaMemset(ctx->d_err, 0, 256); }
  if (e == cudaSuccess) {
    step = "cudaStreamCreate";
    e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) {
    step = "cudaEventCreate";
    e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_info, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) { step = "cudaFuncSetAttribute"; e = init_kernel_attributes(&which); }
  if (e != cudaSuccess) {
    g_create_error = std::string(step) + " " + which + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_info) cudaEventDestroy(ctx->ev_info);
    delete ctx;
    return TR_ERR_CUDA;
  }
  ctx->d_seed = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(ctx->d_err) + 128);
  *out = ctx;
  return TR_OK;
}

void tr_destroy(tr_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->host_stage) cudaFree(ctx->host_stage);
  drop_graph(ctx);
  if (ctx->bexec) cudaGraphExecDestroy(ctx->bexec);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_info) cudaEventDestroy(ctx->ev_info);
  if (ctx->d_err) cudaFree(ctx->d_err);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
}

const char* tr_last_error(const tr_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

tr_status tr_status_sync(tr_ctx* ctx, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  DeviceGuard g(ctx->device);
  return read_device_error(ctx, S(stream));
}

tr_status tr_leverage_planes(tr_ctx* ctx, const float* A_hi, const float* A_lo, int64_t I,
                             int L, double* p, double* cdf, int* branch, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  if (!A_hi || !A_lo || !p || !cdf) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  if (!lev_precond_fits(I, L))
    return fail(ctx, TR_ERR_INVALID_ARG, "tr_leverage_planes needs I >= L, 4 <= L <= 128 "
                "(I=%lld L=%d)", static_cast<long long>(I), L);
  if ((reinterpret_cast<uintptr_t>(A_hi) | reinterpret_cast<uintptr_t>(A_lo)) & 15)
    return fail(ctx, TR_ERR_INVALID_ARG, "A_hi and A_lo must be 16-byte aligned");
  DeviceGuard g(ctx->device);
  const size_t need = leverage_bytes(I, L) + static_cast<size_t>(I) * L * sizeof(double) + 256;
  TR_TRY(ensure_ws(ctx, need));
  cudaStream_t st = S(stream);
  // the FP64 matrix (hi + lo) for the fallback's row solves, after the leverage workspace
  double* mat = reinterpret_cast<double*>(ctx->arena + ((leverage_bytes(I, L) + 255) & ~size_t(255)));
  TR_CUDA(launch_planes_sum(A_hi, A_lo, static_cast<int64_t>(I) * L, mat, st));
  TR_TRY(leverage_dist(ctx, ctx->arena, mat, I, L, p, cdf, nullptr, st, nullptr, true, A_hi,
                       A_lo));
  if (branch) {
    Carver c(ctx->arena);
    LevPass p1{}, p2{};
    double* ell;
    leverage_plan(c, I, L, &p1, &p2, &ell);
    TR_CUDA(launch_copy_int(precond_enabled() ? p1.pre.state : nullptr, 1, branch, st));
  }
  return TR_OK;
}

tr_status tr_leverage(tr_ctx* ctx, const double* core, int64_t I, int Rl, int Rr, double* p,
                      double* cdf, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  if (!core || !p || !cdf) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  if (I < 1 || Rl < 1 || Rr < 1 || Rl * Rr > kMaxL)
    return fail(ctx, TR_ERR_INVALID_ARG, "bad core shape I=%lld Rl=%d Rr=%d",
                static_cast<long long>(I), Rl, Rr);
  DeviceGuard g(ctx->device);
  TR_TRY(ensure_ws(ctx, leverage_bytes(I, Rl * Rr)));
  return leverage_run(ctx, ctx->arena, core, I, Rl, Rr, p, cdf, S(stream));
}

tr_status tr_sample(tr_ctx* ctx, int N, int k, const int64_t* dims, const double* const* p,
                    const double* const* cdf, int64_t J, uint64_t seed, uint64_t update_id,
                    int32_t* idx, double* w, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_shape(ctx, N, dims, nullptr));
  if (k < 0 || k >= N) return fail(ctx, TR_ERR_INVALID_ARG, "k=%d outside [0, N)", k);
  if (J < 1 || J > INT32_MAX) return fail(ctx, TR_ERR_INVALID_ARG, "J=%lld", static_cast<long long>(J));
  if (!p || !cdf || !idx || !w) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  SampleArgs sa{};
  sa.npos = N - 1;
  for (int m = 0; m < N - 1; ++m) {
    const int mode = (k + 1 + m) % N;
    if (!p[mode] || !cdf[mode]) return fail(ctx, TR_ERR_INVALID_ARG, "p/cdf[%d] is NULL", mode);
    sa.p[m] = p[mode];
    sa.cdf[m] = cdf[mode];
    sa.I[m] = dims[mode];
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  TR_LAUNCH("sample", launch_sample(sa, J, seed, update_id, idx, w, st));
  return TR_OK;
}

tr_status tr_sample_uniform(tr_ctx* ctx, int N, int k, const int64_t* dims, int64_t J,
                            uint64_t seed, uint64_t update_id, int32_t* idx, double* w,
                            tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_shape(ctx, N, dims, nullptr));
  if (k < 0 || k >= N) return fail(ctx, TR_ERR_INVALID_ARG, "k=%d outside [0, N)", k);
  if (J < 1 || J > INT32_MAX) return fail(ctx, TR_ERR_INVALID_ARG, "J=%lld", static_cast<long long>(J));
  if (!idx || !w) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  SampleArgs sa{};
  sa.npos = N - 1;
  sa.uniform = 1;
  for (int m = 0; m < N - 1; ++m) sa.I[m] = dims[(k + 1 + m) % N];
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  TR_LAUNCH("sample", launch_sample(sa, J, seed, update_id, idx, w, st));
  return TR_OK;
}

tr_status tr_set_sampling(tr_ctx* ctx, tr_sampling sampling) {
  TR_TRY(check_ctx(ctx));
  if (sampling != TR_SAMPLING_LEVERAGE && sampling != TR_SAMPLING_UNIFORM)
    return fail(ctx, TR_ERR_INVALID_ARG, "sampling=%d is not a tr_sampling value",
                static_cast<int>(sampling));
  ctx->sampling = sampling;
  return TR_OK;
}

tr_status tr_set_ls_rank(tr_ctx* ctx, tr_ls_rank rule) {
  TR_TRY(check_ctx(ctx));
  if (rule != TR_LS_RANK_STOP && rule != TR_LS_RANK_DROP)
    return fail(ctx, TR_ERR_INVALID_ARG, "ls rank rule=%d is not a tr_ls_rank value",
                static_cast<int>(rule));
  ctx->ls_rank = rule;
  return TR_OK;
}

tr_status tr_get_ls_rank(const tr_ctx* ctx, tr_ls_rank* rule) {
  if (!ctx || !rule) return TR_ERR_INVALID_ARG;
  *rule = ctx->ls_rank;
  return TR_OK;
}

tr_status tr_set_factorization(tr_ctx* ctx, tr_factorization f) {
  if (!ctx) return TR_ERR_INVALID_ARG;
  if (f != TR_FACTOR_DEFAULT && f != TR_FACTOR_FP64)
    return fail(ctx, TR_ERR_INVALID_ARG, "unknown factorization %d", static_cast<int>(f));
  ctx->factorization = f;
  return TR_OK;
}

tr_status tr_get_factorization(const tr_ctx* ctx, tr_factorization* f) {
  if (!ctx || !f) return TR_ERR_INVALID_ARG;
  *f = ctx->factorization;
  return TR_OK;
}

tr_status tr_set_wait_limit(tr_ctx* ctx, int64_t polls) {
  if (!ctx) return TR_ERR_INVALID_ARG;
  ctx->wait_limit = polls < 0 ? -1 : static_cast<long long>(polls);
  return TR_OK;
}

tr_status tr_get_wait_limit(const tr_ctx* ctx, int64_t* polls) {
  if (!ctx || !polls) return TR_ERR_INVALID_ARG;
  *polls = ctx->wait_limit;
  return TR_OK;
}

tr_status tr_get_sampling(const tr_ctx* ctx, tr_sampling* sampling) {
  if (!ctx || !sampling) return TR_ERR_INVALID_ARG;
  *sampling = ctx->sampling;
  return TR_OK;
}

tr_status tr_subchain(tr_ctx* ctx, int N, int k, const int64_t* dims, const int* ranks,
                      const double* const* cores, const int32_t* idx, const double* w,
                      int64_t J, void* A, tr_dtype A_dtype, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_shape(ctx, N, dims, ranks));
  if (!ranks) return fail(ctx, TR_ERR_INVALID_ARG, "ranks is NULL");
  if (k < 0 || k >= N) return fail(ctx, TR_ERR_INVALID_ARG, "k=%d outside [0, N)", k);
  if (J < 1) return fail(ctx, TR_ERR_INVALID_ARG, "J=%lld", static_cast<long long>(J));
  if (!cores || !idx || !A) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  if (A_dtype != TR_F32 && A_dtype != TR_F64) return fail(ctx, TR_ERR_INVALID_ARG, "bad dtype");
  ChainArgs ca{};
  ca.npos = N - 1;
  for (int m = 0; m < N - 1; ++m) {
    const int mode = (k + 1 + m) % N;
    if (!cores[mode]) return fail(ctx, TR_ERR_INVALID_ARG, "cores[%d] is NULL", mode);
    ca.core[m] = cores[mode];
    ca.I[m] = dims[mode];
    ca.rl[m] = rl_of(ranks, N, mode);
    ca.rr[m] = ranks[mode];
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  TR_LAUNCH("subchain", launch_subchain(ca, idx, w, J, A, A_dtype == TR_F64, ctx->d_err, st));
  return TR_OK;
}

tr_status tr_gather(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N, const int64_t* dims,
                    int k, const int32_t* idx, const double* w, int64_t J, void* Y,
                    tr_dtype Y_dtype, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_shape(ctx, N, dims, nullptr));
  if (k < 0 || k >= N) return fail(ctx, TR_ERR_INVALID_ARG, "k=%d outside [0, N)", k);
  if (J < 1) return fail(ctx, TR_ERR_INVALID_ARG, "J=%lld", static_cast<long long>(J));
  if (!X || !idx || !Y) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  if ((X_dtype != TR_F32 && X_dtype != TR_F64) || (Y_dtype != TR_F32 && Y_dtype != TR_F64))
    return fail(ctx, TR_ERR_INVALID_ARG, "bad dtype");
  int64_t stride[kMaxModes];
  row_major_strides(N, dims, stride);
  GatherArgs ga{};
  ga.npos = N - 1;
  for (int m = 0; m < N - 1; ++m) {
    const int mode = (k + 1 + m) % N;
    ga.I[m] = dims[mode];
    ga.stride[m] = stride[mode];
  }
  ga.In = dims[k];
  ga.stride_n = stride[k];
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  TR_LAUNCH("gather", launch_gather(ga, X, X_dtype == TR_F64, idx, w, J, Y, Y_dtype == TR_F64,
                                    ctx->d_err, st));
  return TR_OK;
}

tr_status tr_solve(tr_ctx* ctx, const void* A, const void* Y, tr_dtype dtype, int64_t J, int Rl,
                   int Rr, int64_t I, tr_precision prec, double* core_out, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  if (!A || !Y || !core_out) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  if (J < 1 || I < 1 || Rl < 1 || Rr < 1 || Rl * Rr > kMaxL)
    return fail(ctx, TR_ERR_INVALID_ARG, "bad sizes J=%lld L=%d I=%lld",
                static_cast<long long>(J), Rl * Rr, static_cast<long long>(I));
  if (prec == TR_PREC_FP64 && dtype != TR_F64)
    return fail(ctx, TR_ERR_INVALID_ARG, "TR_PREC_FP64 needs FP64 A and Y");
  if (prec == TR_PREC_MIXED && dtype != TR_F32)
    return fail(ctx, TR_ERR_INVALID_ARG, "TR_PREC_MIXED needs FP32 A and Y");
  if (prec != TR_PREC_FP64 && prec != TR_PREC_MIXED)
    return fail(ctx, TR_ERR_INVALID_ARG, "bad precision");
  const bool f64 = prec == TR_PREC_FP64;
  DeviceGuard g(ctx->device);
  TR_TRY(ensure_ws(ctx, solve_bytes(J, Rl * Rr, I, f64)));
  return solve_run(ctx, ctx->arena, A, Y, f64, J, Rl, Rr, I, !f64, core_out, S(stream));
}

tr_status tr_init_cores(tr_ctx* ctx, int N, const int64_t* dims, const int* ranks, uint64_t seed,
                        int k_begin, double* const* cores, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_shape(ctx, N, dims, ranks));
  if (!ranks || !cores) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  for (int k = k_begin < 0 ? 0 : k_begin; k < N; ++k) {
    if (!cores[k]) return fail(ctx, TR_ERR_INVALID_ARG, "cores[%d] is NULL", k);
    const int64_t count = dims[k] * rl_of(ranks, N, k) * ranks[k];
    TR_LAUNCH("init_normal", launch_init_normal(cores[k], count, seed, static_cast<uint32_t>(k),
                                                nullptr, st));
  }
  return TR_OK;
}

static tr_status check_als(tr_ctx* ctx, const void* X, tr_dtype xdt, int N, const int64_t* dims,
                           const int* ranks, int64_t J, int sweeps, tr_precision prec,
                           double* const* cores, const double* const* init) {
  TR_TRY(check_shape(ctx, N, dims, ranks));
  if (!ranks) return fail(ctx, TR_ERR_INVALID_ARG, "ranks is NULL");
  if (!X || !cores) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  for (int k = 0; k < N; ++k)
    if (!cores[k]) return fail(ctx, TR_ERR_INVALID_ARG, "cores[%d] is NULL", k);
  if (J < 1 || J > INT32_MAX) return fail(ctx, TR_ERR_INVALID_ARG, "J=%lld", static_cast<long long>(J));
  if (sweeps < 0) return fail(ctx, TR_ERR_INVALID_ARG, "sweeps=%d", sweeps);
  if (xdt != TR_F32 && xdt != TR_F64) return fail(ctx, TR_ERR_INVALID_ARG, "bad X dtype");
  if (prec != TR_PREC_FP64 && prec != TR_PREC_MIXED)
    return fail(ctx, TR_ERR_INVALID_ARG, "bad precision");
  if (init)
    for (int k = 1; k < N; ++k)
      if (!init[k]) return fail(ctx, TR_ERR_INVALID_ARG, "init_cores[%d] is NULL", k);
  return TR_OK;
}

tr_status tr_als_sampled(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N, const int64_t* dims,
                         const int* ranks, int64_t J, int sweeps, uint64_t seed,
                         tr_precision prec, const double* const* init_cores,
                         double* const* cores, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_als(ctx, X, X_dtype, N, dims, ranks, J, sweeps, prec, cores, init_cores));
  DeviceGuard g(ctx->device);
  AlsPlan P{X, X_dtype, N, dims, ranks, J, sweeps, prec, init_cores, cores};
  TR_TRY(als_run(ctx, P, seed, S(stream)));
  tr_status s = read_device_error(ctx, S(stream));
  TR_TRY(fold_graph_marks(ctx));
  return s;
}

tr_status tr_als_sampled_schedule(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N,
                                  const int64_t* dims, const int* ranks,
                                  const int64_t* J_per_sweep, int sweeps, uint64_t seed,
                                  tr_precision prec, const double* const* init_cores,
                                  double* const* cores, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  if (!J_per_sweep && sweeps > 0) return fail(ctx, TR_ERR_INVALID_ARG, "J_per_sweep is NULL");
  int64_t Jmax = 1;
  for (int s = 0; s < sweeps; ++s) {
    if (J_per_sweep[s] < 1 || J_per_sweep[s] > INT32_MAX)
      return fail(ctx, TR_ERR_INVALID_ARG, "J_per_sweep[%d]=%lld", s,
                  static_cast<long long>(J_per_sweep[s]));
    Jmax = J_per_sweep[s] > Jmax ? J_per_sweep[s] : Jmax;
  }
  TR_TRY(check_als(ctx, X, X_dtype, N, dims, ranks, Jmax, sweeps, prec, cores, init_cores));
  DeviceGuard g(ctx->device);
  AlsPlan P{X, X_dtype, N, dims, ranks, Jmax, sweeps, prec, init_cores, cores};
  P.Js = J_per_sweep;
  TR_TRY(als_run(ctx, P, seed, S(stream)));
  tr_status st = read_device_error(ctx, S(stream));
  TR_TRY(fold_graph_marks(ctx));
  return st;
}

tr_status tr_als_sampled_adaptive(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N,
                                  const int64_t* dims, const int* ranks,
                                  const int64_t* J_per_update, int sweeps, uint64_t seed,
                                  tr_precision prec, const double* const* init_cores,
                                  double* const* cores, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  if (!J_per_update && sweeps > 0) return fail(ctx, TR_ERR_INVALID_ARG, "J_per_update is NULL");
  TR_TRY(check_shape(ctx, N, dims, ranks));
  int64_t Jmax = 1;
  for (int64_t e = 0; e < static_cast<int64_t>(sweeps) * N; ++e) {
    if (J_per_update[e] < 1 || J_per_update[e] > INT32_MAX)
      return fail(ctx, TR_ERR_INVALID_ARG, "J_per_update[%lld]=%lld", static_cast<long long>(e),
                  static_cast<long long>(J_per_update[e]));
    Jmax = J_per_update[e] > Jmax ? J_per_update[e] : Jmax;
  }
  TR_TRY(check_als(ctx, X, X_dtype, N, dims, ranks, Jmax, sweeps, prec, cores, init_cores));
  DeviceGuard g(ctx->device);
  AlsPlan P{X, X_dtype, N, dims, ranks, Jmax, sweeps, prec, init_cores, cores};
  P.Jupd = J_per_update;
  TR_TRY(als_run(ctx, P, seed, S(stream)));
  tr_status st = read_device_error(ctx, S(stream));
  TR_TRY(fold_graph_marks(ctx));
  return st;
}

tr_status tr_set_merge_duplicates(tr_ctx* ctx, int on) {
  if (!ctx) return TR_ERR_INVALID_ARG;
  ctx->merge = on ? 1 : 0;
  return TR_OK;
}

tr_status tr_get_merge_duplicates(const tr_ctx* ctx, int* on) {
  if (!ctx || !on) return TR_ERR_INVALID_ARG;
  *on = ctx->merge;
  return TR_OK;
}

tr_status tr_merge_samples(tr_ctx* ctx, int N, int k, const int64_t* dims, const int32_t* idx,
                           const double* w, int64_t J, int32_t* idx_out, double* w_out,
                           int64_t* J_out, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_shape(ctx, N, dims, nullptr));
  if (k < 0 || k >= N) return fail(ctx, TR_ERR_INVALID_ARG, "k=%d outside [0, N)", k);
  if (!idx || !w || !idx_out || !w_out || !J_out)
    return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  int64_t I[kMaxModes];
  for (int m = 0; m < N - 1; ++m) I[m] = dims[(k + 1 + m) % N];
  MergeArgs ma{};
  if (!merge_fits(J, N - 1, I, &ma))
    return fail(ctx, TR_ERR_INVALID_ARG,
                "J=%lld outside [1, %d] or the sampled index space is 2^63 or larger",
                static_cast<long long>(J), kMergeMaxJ);
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  TR_LAUNCH("merge", launch_merge(idx, w, J, N - 1, ma, idx_out, w_out, J_out, st));
  return TR_OK;
}

tr_status tr_als(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N, const int64_t* dims,
                 const int* ranks, int sweeps, uint64_t seed, tr_precision prec,
                 const double* const* init_cores, double* const* cores, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_als(ctx, X, X_dtype, N, dims, ranks, 1, sweeps, prec, cores, init_cores));
  const bool f64 = prec == TR_PREC_FP64, x64 = X_dtype == TR_F64;
  const size_t es = f64 ? 8 : 4;
  // rows of each update: every multi-index of the other modes
  std::vector<int64_t> P(N, 1);
  int64_t numel = 1, Pmax = 0;
  int Lmax = 0;
  for (int k = 0; k < N; ++k) numel *= dims[k];
  for (int n = 0; n < N; ++n) {
    P[n] = numel / dims[n];
    Pmax = P[n] > Pmax ? P[n] : Pmax;
    const int L = rl_of(ranks, N, n) * ranks[n];
    Lmax = L > Lmax ? L : Lmax;
    if (dims[n] > 65535LL * 32)
      return fail(ctx, TR_ERR_INVALID_ARG, "dims[%d]=%lld exceeds 2097120 (dense unfolding)", n,
                  static_cast<long long>(dims[n]));
  }
  Carver dry(nullptr);
  dry.take<int32_t>(static_cast<size_t>(Pmax) * (N - 1));
  dry.take<char>(static_cast<size_t>(Pmax) * Lmax * es);
  dry.take<char>(static_cast<size_t>(numel) * es);
  const size_t persist = (dry.off + 255) & ~size_t(255);
  size_t solve_max = 0;
  for (int n = 0; n < N; ++n) {
    const size_t b = solve_bytes(P[n], rl_of(ranks, N, n) * ranks[n], dims[n], f64);
    solve_max = b > solve_max ? b : solve_max;
  }
  DeviceGuard g(ctx->device);
  TR_TRY(ensure_ws(ctx, persist + solve_max + 256));
  Carver c(ctx->arena);
  int32_t* idx = c.take<int32_t>(static_cast<size_t>(Pmax) * (N - 1));
  void* A = c.take<char>(static_cast<size_t>(Pmax) * Lmax * es);
  void* Y = c.take<char>(static_cast<size_t>(numel) * es);
  char* ws = ctx->arena + persist;
  cudaStream_t st = S(stream);
  for (int k = 1; k < N; ++k) {
    const size_t count = static_cast<size_t>(dims[k]) * rl_of(ranks, N, k) * ranks[k];
    if (init_cores) {
      TR_CUDA(cudaMemcpyAsync(cores[k], init_cores[k], count * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
    } else {
      TR_LAUNCH("init_normal", launch_init_normal(cores[k], static_cast<int64_t>(count), seed,
                                                  static_cast<uint32_t>(k), nullptr, st));
    }
  }
  DenseDims dd{};
  for (int k = 0; k < N; ++k) dd.I[k] = dims[k];
  for (int s = 0; s < sweeps; ++s) {
    for (int n = 0; n < N; ++n) {
      ChainArgs ca{};
      ca.npos = N - 1;
      for (int m = 0; m < N - 1; ++m) {
        const int mode = (n + 1 + m) % N;
        ca.core[m] = cores[mode];
        ca.I[m] = dims[mode];
        ca.rl[m] = rl_of(ranks, N, mode);
        ca.rr[m] = ranks[mode];
      }
      TR_LAUNCH("enumerate", launch_enumerate(N, n, dd, idx, st));
      TR_LAUNCH("subchain", launch_subchain(ca, idx, nullptr, P[n], A, f64, ctx->d_err, st));
      // the last mode's rows are X itself when X already has the LS step's type
      const void* Yn = (n == N - 1 && x64 == f64) ? X : Y;
      if (Yn == Y) TR_LAUNCH("unfold", launch_unfold(X, x64, N, n, dd, Y, f64, st));
      TR_TRY(update_run(ctx, ws, solve_max, A, Yn, f64, P[n], rl_of(ranks, N, n), ranks[n],
                        dims[n], cores[n], nullptr, nullptr, st, ctx->side));
    }
  }
  return read_device_error(ctx, st);
}

tr_status tr_als_sampled_host(tr_ctx* ctx, const void* X_host, tr_dtype X_dtype, int N,
                              const int64_t* dims, const int* ranks, int64_t J, int sweeps,
                              uint64_t seed, tr_precision prec,
                              const double* const* init_cores_host, double* const* cores_host,
                              tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_als(ctx, X_host, X_dtype, N, dims, ranks, J, sweeps, prec, cores_host,
                   init_cores_host));
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  int64_t numel = 1;
  for (int k = 0; k < N; ++k) numel *= dims[k];
  const size_t xbytes = static_cast<size_t>(numel) * (X_dtype == TR_F64 ? 8 : 4);
  std::vector<size_t> cbytes(N);
  size_t total = (xbytes + 255) & ~size_t(255);
  for (int k = 0; k < N; ++k) {
    cbytes[k] = static_cast<size_t>(dims[k]) * rl_of(ranks, N, k) * ranks[k] * sizeof(double);
    total += 2 * ((cbytes[k] + 255) & ~size_t(255));
  }
  if (total > ctx->host_stage_bytes) {
    if (ctx->budget && total + ctx->arena_bytes > ctx->budget)
      return fail(ctx, TR_ERR_BUDGET, "host staging of %zu bytes exceeds the HBM budget", total);
    TR_CUDA(cudaDeviceSynchronize());
    if (ctx->host_stage) cudaFree(ctx->host_stage);
    ctx->host_stage = nullptr;
    ctx->host_stage_bytes = 0;
    if (cudaMalloc(&ctx->host_stage, total) != cudaSuccess) {
      cudaGetLastError();
      ctx->host_stage = nullptr;
      return fail(ctx, TR_ERR_OOM, "cudaMalloc of %zu staging bytes failed", total);
    }
    ctx->host_stage_bytes = total;
  }
  char* base = ctx->host_stage;
  void* dX = base;
  size_t off = (xbytes + 255) & ~size_t(255);
  std::vector<double*> dcores(N), dinit(N, nullptr);
  for (int k = 0; k < N; ++k) {
    dcores[k] = reinterpret_cast<double*>(base + off);
    off += (cbytes[k] + 255) & ~size_t(255);
    dinit[k] = reinterpret_cast<double*>(base + off);
    off += (cbytes[k] + 255) & ~size_t(255);
  }
  TR_CUDA(cudaMemcpyAsync(dX, X_host, xbytes, cudaMemcpyHostToDevice, st));
  if (init_cores_host) {
    for (int k = 1; k < N; ++k) {
      if (!init_cores_host[k]) return fail(ctx, TR_ERR_INVALID_ARG, "init_cores[%d] is NULL", k);
      TR_CUDA(cudaMemcpyAsync(dinit[k], init_cores_host[k], cbytes[k], cudaMemcpyHostToDevice, st));
    }
  }
  AlsPlan P{dX, X_dtype, N, dims, ranks, J, sweeps, prec,
            init_cores_host ? dinit.data() : nullptr, dcores.data()};
  TR_TRY(als_run(ctx, P, seed, st));
  for (int k = 0; k < N; ++k)
    TR_CUDA(cudaMemcpyAsync(cores_host[k], dcores[k], cbytes[k], cudaMemcpyDeviceToHost, st));
  tr_status s = read_device_error(ctx, st);
  TR_TRY(fold_graph_marks(ctx));
  return s;
}

tr_status tr_als_sampled_batched(tr_ctx* ctx, const tr_instance* inst, int count,
                                 tr_dtype X_dtype, int sweeps, tr_precision prec,
                                 tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  if (!inst || count < 1) return fail(ctx, TR_ERR_INVALID_ARG, "no instances");
  if (sweeps < 0) return fail(ctx, TR_ERR_INVALID_ARG, "sweeps=%d", sweeps);
  if (X_dtype != TR_F32 && X_dtype != TR_F64) return fail(ctx, TR_ERR_INVALID_ARG, "bad X dtype");
  if (prec != TR_PREC_FP64 && prec != TR_PREC_MIXED)
    return fail(ctx, TR_ERR_INVALID_ARG, "bad precision");
  const bool f64 = prec == TR_PREC_FP64;
  for (int i = 0; i < count; ++i) {
    const tr_instance& in = inst[i];
    TR_TRY(check_shape(ctx, in.N, in.dims, in.ranks));
    if (!in.X) return fail(ctx, TR_ERR_INVALID_ARG, "instance %d: X is NULL", i);
    if (in.J < 1 || in.J > INT32_MAX)
      return fail(ctx, TR_ERR_INVALID_ARG, "instance %d: J=%lld", i, static_cast<long long>(in.J));
    for (int k = 0; k < in.N; ++k)
      if (!in.cores[k]) return fail(ctx, TR_ERR_INVALID_ARG, "instance %d: cores[%d] is NULL", i, k);
  }
  DeviceGuard g(ctx->device);
  cudaStream_t st = S(stream);
  // sizes
  Carver dry(nullptr);
  dry.take<BInst>(count);
  dry.take<unsigned>(count);
  std::vector<BInst> tab(count);
  for (int i = 0; i < count; ++i)
    carve_instance(dry, inst[i].N, inst[i].dims, inst[i].ranks, inst[i].J, f64, tab[i]);
  TR_TRY(ensure_ws(ctx, dry.off));
  Carver c(ctx->arena);
  BInst* dtab = c.take<BInst>(count);
  unsigned* counters = c.take<unsigned>(count);
  BLaunch bl{};
  bl.tab = dtab;
  bl.count = count;
  bl.f64 = f64;
  bl.xf64 = X_dtype == TR_F64;
  bl.spw = ctx->tiles.samples_per_warp;
  bl.ctile = ctx->tiles.contract_tile;
  bl.leverage = ctx->sampling == TR_SAMPLING_LEVERAGE;
  bl.ls_mode = ctx->ls_rank == TR_LS_RANK_DROP ? 1 : 0;
  int nmax_modes = 0, steps = 0;
  bool draw = false;
  for (int i = 0; i < count; ++i) {
    const tr_instance& in = inst[i];
    BInst& d = tab[i];
    d = BInst{};
    carve_instance(c, in.N, in.dims, in.ranks, in.J, f64, d);
    d.X = in.X;
    d.N = in.N;
    d.xf64 = X_dtype == TR_F64;
    d.nupd = sweeps * in.N;
    d.draw_init = in.init_given ? 0 : 1;
    d.uniform = bl.leverage ? 0 : 1;
    d.J = in.J;
    d.seed = in.seed;
    row_major_strides(in.N, in.dims, d.stride);
    for (int k = 0; k < in.N; ++k) {
      d.dims[k] = in.dims[k];
      d.ranks[k] = in.ranks[k];
      d.cores[k] = in.cores[k];
    }
    d.counter = counters + i;
    const BSizes z = bsizes(in.N, in.dims, in.ranks);
    bl.Jmax = in.J > bl.Jmax ? in.J : bl.Jmax;
    bl.Lmax = z.Lmax > bl.Lmax ? z.Lmax : bl.Lmax;
    bl.Imax = z.Imax > bl.Imax ? z.Imax : bl.Imax;
    bl.n1max = z.n1 > bl.n1max ? z.n1 : bl.n1max;
    bl.n2max = z.n2 > bl.n2max ? z.n2 : bl.n2max;
    nmax_modes = in.N > nmax_modes ? in.N : nmax_modes;
    steps = d.nupd > steps ? d.nupd : steps;
    draw = draw || d.draw_init;
  }
  ctx->btab = tab;
  TR_CUDA(cudaMemcpyAsync(dtab, ctx->btab.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice,
                          st));
  TR_CUDA(cudaMemsetAsync(counters, 0, sizeof(unsigned) * count, st));
  if (!graphs_enabled()) {
    TR_TRY(batched_issue(ctx, bl, nmax_modes, steps, draw, st));
  } else {
    std::vector<uint64_t> key = {static_cast<uint64_t>(count), static_cast<uint64_t>(bl.Jmax),
                                 static_cast<uint64_t>(bl.Lmax), static_cast<uint64_t>(bl.Imax),
                                 static_cast<uint64_t>(bl.n1max), static_cast<uint64_t>(bl.n2max),
                                 static_cast<uint64_t>(f64), static_cast<uint64_t>(bl.xf64),
                                 static_cast<uint64_t>(nmax_modes), static_cast<uint64_t>(steps),
                                 static_cast<uint64_t>(draw), reinterpret_cast<uintptr_t>(dtab),
                                 static_cast<uint64_t>(ctx->prof),
                                 static_cast<uint64_t>(bl.spw), static_cast<uint64_t>(bl.ctile),
                                 static_cast<uint64_t>(bl.leverage),
                                 static_cast<uint64_t>(bl.ls_mode)};
    if (!ctx->bexec || key != ctx->bkey) {
      if (ctx->bexec) cudaGraphExecDestroy(ctx->bexec);
      ctx->bexec = nullptr;
      cudaGraph_t gr = nullptr;
      const bool prof = ctx->prof;
      ctx->prof = false;   // no profiler events inside the batched graph
      TR_CUDA(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
      tr_status s2 = batched_issue(ctx, bl, nmax_modes, steps, draw, ctx->cap);
      cudaError_t e = cudaStreamEndCapture(ctx->cap, &gr);
      ctx->prof = prof;
      if (s2 != TR_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s2;
      }
      if (e != cudaSuccess)
        return fail(ctx, TR_ERR_CUDA, "batched graph capture failed: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&ctx->bexec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) {
        ctx->bexec = nullptr;
        return fail(ctx, TR_ERR_CUDA, "batched graph instantiation failed: %s",
                    cudaGetErrorString(e));
      }
      ctx->bkey = key;
    }
    TR_CUDA(cudaGraphLaunch(ctx->bexec, st));
  }
  return read_device_error(ctx, st);
}

tr_status tr_set_batched_tiles(tr_ctx* ctx, const tr_batched_tiles* tiles) {
  TR_TRY(check_ctx(ctx));
  if (!tiles) return fail(ctx, TR_ERR_INVALID_ARG, "tiles is NULL");
  if (tiles->samples_per_warp < 1 || tiles->samples_per_warp > 8)
    return fail(ctx, TR_ERR_INVALID_ARG, "samples_per_warp=%d outside [1, 8]",
                tiles->samples_per_warp);
  if (tiles->contract_tile != 64 && tiles->contract_tile != 32)
    return fail(ctx, TR_ERR_INVALID_ARG, "contract_tile=%d is not 64 or 32",
                tiles->contract_tile);
  ctx->tiles = *tiles;
  return TR_OK;
}

tr_status tr_get_batched_tiles(const tr_ctx* ctx, tr_batched_tiles* tiles) {
  if (!ctx || !tiles) return TR_ERR_INVALID_ARG;
  *tiles = ctx->tiles;
  return TR_OK;
}

tr_status tr_rel_error(tr_ctx* ctx, const void* X, tr_dtype X_dtype, int N, const int64_t* dims,
                       const int* ranks, const double* const* cores, double* rel_err,
                       tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  TR_TRY(check_shape(ctx, N, dims, ranks));
  if (!ranks || !X || !cores || !rel_err) return fail(ctx, TR_ERR_INVALID_ARG, "null pointer");
  if (X_dtype != TR_F32 && X_dtype != TR_F64) return fail(ctx, TR_ERR_INVALID_ARG, "bad dtype");
  FitArgs fa{};
  fa.N = N;
  for (int k = 0; k < N; ++k) {
    if (!cores[k]) return fail(ctx, TR_ERR_INVALID_ARG, "cores[%d] is NULL", k);
    fa.core[k] = cores[k];
    fa.dims[k] = dims[k];
    fa.ranks[k] = ranks[k];
  }
  DeviceGuard g(ctx->device);
  int blocks;
  const bool xf64 = X_dtype == TR_F64;
  const size_t bytes = fit_workspace(fa, xf64, &blocks);
  TR_TRY(ensure_ws(ctx, bytes));
  double* partial = reinterpret_cast<double*>(ctx->arena);
  cudaStream_t st = S(stream);
  TR_LAUNCH("fit", launch_fit(fa, X, xf64, ctx->arena, blocks, ctx->d_err, st));
  std::vector<double> h(2 * static_cast<size_t>(blocks));
  TR_CUDA(cudaMemcpyAsync(h.data(), partial, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  TR_TRY(read_device_error(ctx, st));
  double se = 0.0, sx = 0.0;
  for (int b = 0; b < blocks; ++b) { se += h[b]; sx += h[blocks + b]; }
  *rel_err = sx > 0.0 ? std::sqrt(se / sx) : (se > 0.0 ? INFINITY : 0.0);
  return TR_OK;
}

tr_status tr_profile_begin(tr_ctx* ctx) {
  TR_TRY(check_ctx(ctx));
  ctx->prof = true;
  ctx->ev_used = 0;
  ctx->prof_marks.clear();
  ctx->prof_tot.clear();
  ctx->prof_snapshot.clear();
  return TR_OK;
}

tr_status tr_profile_end(tr_ctx* ctx, tr_stream stream) {
  TR_TRY(check_ctx(ctx));
  DeviceGuard g(ctx->device);
  ctx->prof = false;
  TR_CUDA(cudaStreamSynchronize(S(stream)));
  TR_CUDA(cudaDeviceSynchronize());
  for (const auto& m : ctx->prof_marks) {
    float ms = 0.f;
    TR_CUDA(cudaEventElapsedTime(&ms, ctx->ev_pool[m.second], ctx->ev_pool[m.second + 1]));
    add_prof(ctx, m.first, ms);
  }
  ctx->prof_marks.clear();
  ctx->ev_used = 0;
  ctx->prof_snapshot.assign(ctx->prof_tot.begin(), ctx->prof_tot.end());
  return TR_OK;
}

int tr_profile_count(const tr_ctx* ctx) {
  return ctx ? static_cast<int>(ctx->prof_snapshot.size()) : 0;
}

tr_status tr_profile_entry(const tr_ctx* ctx, int i, const char** name, double* total_ms,
                           int64_t* launches) {
  if (!ctx || i < 0 || i >= static_cast<int>(ctx->prof_snapshot.size()))
    return TR_ERR_INVALID_ARG;
  const auto& e = ctx->prof_snapshot[i];
  if (name) *name = e.first.c_str();
  if (total_ms) *total_ms = e.second.first;
  if (launches) *launches = e.second.second;
  return TR_OK;
}

}  // extern "C"

namespace trk {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace trk
