// Batched stages of TR-ALS-Sampled (Alg. 2 per instance, Alg. 3 + Alg. 4 for the sketch):
// one launch per stage for every instance of the table; see batched.cuh.
#include "batched.cuh"
#include "cholesky_body.cuh"
#include "draw.cuh"
#include "fit_tc.cuh"
#include "trsm_body.cuh"

namespace trk {
namespace {

// The core being updated (or, in an initialisation step, the core whose initial distribution
// is formed) and its sizes. Leverage stages (`lev`) run in both kinds of step; the sampling
// and solve stages only in updates.
struct Cur {
  bool active;
  bool init;
  int n, Rl, Rr, L;
  int64_t I;
  int t;             // update id (step) of an update
};

__device__ __forceinline__ Cur current(const BInst& d, int step, int init_k, bool lev) {
  Cur c{};
  if (lev && d.uniform) return c;   // uniform sampling forms no distributions
  int k = 0, t = step;
  if (d.slot) {
    const SlotState& s = *d.slot;
    if (s.status != kSlotRunning) return c;
    t = s.step;
    if (t < 0) {
      if (!lev) return c;
      k = t + d.N;
    }
  } else if (init_k > 0) {
    if (d.nupd <= 0 || init_k >= d.N) return c;
    k = init_k;
  }
  if (k > 0) {
    c.init = true;
    c.n = k;
  } else {
    if (t >= d.nupd) return c;
    c.n = t % d.N;
    c.t = t;
  }
  c.active = true;
  c.Rl = d.ranks[(c.n - 1 + d.N) % d.N];
  c.Rr = d.ranks[c.n];
  c.L = c.Rl * c.Rr;
  c.I = d.dims[c.n];
  return c;
}

// ------------------------------------------------------------------------------------
// Initial cores N(0,1) (same stream as launch_init_normal: stream id = core index).
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) kb_init_cores(const BInst* __restrict__ tab) {
  const BInst& d = tab[blockIdx.x];
  if (!d.draw_init) return;
  if (d.slot) {
    if (d.slot->status != kSlotRunning || d.slot->step != 1 - d.N) return;
  } else if (d.nupd <= 0) {
    return;
  }
  const uint32_t k0 = static_cast<uint32_t>(d.seed), k1 = static_cast<uint32_t>(d.seed >> 32);
  for (int k = 1; k < d.N; ++k) {
    const int64_t count = d.dims[k] * d.ranks[(k - 1 + d.N) % d.N] * d.ranks[k];
    const int64_t pairs = (count + 1) / 2;
    double* out = d.cores[k];
    for (int64_t q = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x; q < pairs;
         q += static_cast<int64_t>(gridDim.y) * blockDim.x) {
      double z0, z1;
      normal_pair(q, static_cast<uint32_t>(k), k0, k1, &z0, &z1);
      out[2 * q] = z0;
      if (2 * q + 1 < count) out[2 * q + 1] = z1;
    }
  }
}

// ------------------------------------------------------------------------------------
// Draws (Alg. 3), sampled subchain rows (Alg. 4) and sampled fibres (Alg. 2) for one chunk
// of one instance's samples: one warp per sample.
// ------------------------------------------------------------------------------------
constexpr int SW = 8;     // warps per CTA
constexpr int kSpwMax = 8;   // samples per warp: a launch parameter in [1, 8] (tiles)

template <typename T, typename TX>
__global__ void __launch_bounds__(SW * 32) kb_sample(const BInst* __restrict__ tab, int step,
                                                     int spw) {
  __shared__ T sS[SW][kMaxL];
  __shared__ T sG[SW][kMaxL];
  __shared__ ChainArgs ca;
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, 0, false);
  if (!cu.active) return;
  const int64_t j0 = static_cast<int64_t>(blockIdx.y) * SW * spw;
  if (j0 >= d.J) return;
  const int N = d.N, npos = N - 1, n = cu.n;
  if (threadIdx.x == 0) {
    ca.npos = npos;
    for (int m = 0; m < npos; ++m) {
      const int mode = (n + 1 + m) % N;
      ca.core[m] = d.cores[mode];
      ca.I[m] = d.dims[mode];
      ca.rl[m] = d.ranks[(mode - 1 + N) % N];
      ca.rr[m] = d.ranks[mode];
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t k0 = static_cast<uint32_t>(d.seed), k1 = static_cast<uint32_t>(d.seed >> 32);
  const uint32_t u0 = static_cast<uint32_t>(cu.t), u1 = 0u;
  const int mode_l = (lane < npos) ? (n + 1 + lane) % N : 0;
  const TX* __restrict__ X = static_cast<const TX*>(d.X);
  T* A = static_cast<T*>(d.A);
  T* Y = static_cast<T*>(d.Y);
  const int L = cu.L;
  const int64_t I = cu.I, sn = d.stride[n];
  const double wuni = d.uniform ? uniform_weight(d.J, ca.I, npos) : 0.0;
  for (int s = 0; s < spw; ++s) {
    const int64_t j = j0 + warp * spw + s;
    if (j >= d.J) break;
    int64_t mine = 0;
    double pmine = 1.0;
    int64_t off = 0;
    if (lane < npos) {
      const double u = draw_uniform(j, lane, k0, k1, u0, u1);
      if (d.uniform) {
        mine = uniform_index(d.dims[mode_l], u);
      } else {
        mine = inverse_cdf(d.cdf[mode_l], d.p[mode_l], d.dims[mode_l], u);
        pmine = d.p[mode_l][mine];
      }
      off = mine * d.stride[mode_l];
    }
    double wj = wuni;
    if (!d.uniform) {
      double pm[kMaxModes];
      for (int m = 0; m < npos; ++m) pm[m] = __shfl_sync(0xffffffffu, pmine, m);
      wj = sample_weight(d.J, pm, npos);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    auto index = [&](int m) -> int64_t {
      return static_cast<int64_t>(__shfl_sync(0xffffffffu, static_cast<int>(mine), m));
    };
    warp_slice_chain<T>(ca, index, sS[warp], sG[warp], lane);
    const T scale = static_cast<T>(wj);
    for (int e = lane; e < L; e += 32) A[j * L + e] = sS[warp][e] * scale;
    const TX* src = X + off;
    for (int64_t e = lane; e < I; e += 32)
      Y[j * I + e] = static_cast<T>(static_cast<T>(src[e * sn]) * scale);
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// Normal equations C = A^T [A | Y] per instance, square output tiles over all samples
// (no split: one fixed summation order per entry); M = C[:, :L], B^T = C[:, L:]^T in FP64.
// ------------------------------------------------------------------------------------
// TILE x TILE outputs per CTA, 4 x 4 per thread; every entry is summed over the samples in
// the same order for either tile, so the tile (a launch parameter) never changes results.
constexpr int BK = 16;

template <typename T, int TILE>
__global__ void __launch_bounds__((TILE / 4) * (TILE / 4)) kb_contract(
    const BInst* __restrict__ tab, int step) {
  constexpr int BM = TILE, BN = TILE, TXN = TILE / 4, CT = TXN * TXN;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, 0, false);
  if (!cu.active) return;
  const int L = cu.L;
  const int64_t I = cu.I, ldc = L + I;
  const int ntr = (L + BM - 1) / BM;
  const int ntc = static_cast<int>((ldc + BN - 1) / BN);
  const int t = blockIdx.y;
  if (t >= ntr * ntc) return;
  const int r0 = (t / ntc) * BM;
  const int64_t c0 = static_cast<int64_t>(t % ntc) * BN;
  const T* __restrict__ A = static_cast<const T*>(d.A);
  const T* __restrict__ Y = static_cast<const T*>(d.Y);
  const int64_t J = d.J;
  const int tx = threadIdx.x % TXN, ty = threadIdx.x / TXN;
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  for (int64_t jb = 0; jb < J; jb += BK) {
#pragma unroll
    for (int q = 0; q < (BK * BM) / CT; ++q) {
      const int e = threadIdx.x + q * CT;
      const int kk = e / BM, col = e % BM;
      const int64_t j = jb + kk;
      const int r = r0 + col;
      As[kk][col] = (j < J && r < L) ? A[j * L + r] : T(0);
      const int64_t c = c0 + col;
      T b = T(0);
      if (j < J) {
        if (c < L) b = A[j * L + c];
        else if (c < ldc) b = Y[j * I + (c - L)];
      }
      Bs[kk][col] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + TXN * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx + TXN * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = r0 + ty + TXN * u;
    if (r >= L) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t c = c0 + tx + TXN * v;
      if (c < L) d.M[static_cast<int64_t>(r) * L + c] = static_cast<double>(acc[u][v]);
      else if (c < ldc) d.BT[(c - L) * L + r] = static_cast<double>(acc[u][v]);
    }
  }
}

// ------------------------------------------------------------------------------------
// Gram matrices of the leverage passes (FP64, full square, 32 x 32 tiles over all rows).
//   pass 1, tall (I >= L): G1 = S^T S (L x L); wide: G1 = S S^T (I x I), S = the I x L rows
//           (the core at initialisation, B^T during the updates);
//   pass 2 (wide modes only): G2 = C^T C (I x I), C = the pass-1 factor.
// ------------------------------------------------------------------------------------
constexpr int GT = 32, GK = 32, GNT = 256;

__global__ void __launch_bounds__(GNT) kb_gram(const BInst* __restrict__ tab, int step, int init_k,
                                               int pass) {
  __shared__ double P[GK][GT + 1];
  __shared__ double Q[GK][GT + 1];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, true);
  if (!cu.active) return;
  const bool tall = cu.I >= cu.L;
  if (pass == 2 && tall) return;
  const double* S = cu.init ? d.cores[cu.n] : d.BT;
  const double* src;
  int64_t K, lda;
  int n;
  bool trans;
  double* G;
  if (pass == 1) {
    src = S; lda = cu.L; G = d.G1;
    if (tall) { n = cu.L; K = cu.I; trans = false; }
    else { n = static_cast<int>(cu.I); K = cu.L; trans = true; }
  } else {
    src = d.L1row; lda = cu.I; G = d.G2;
    n = static_cast<int>(cu.I); K = cu.I; trans = false;
  }
  const int nt = (n + GT - 1) / GT;
  const int t = blockIdx.y;
  if (t >= nt * nt) return;
  const int p0 = (t / nt) * GT, q0 = (t % nt) * GT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t kb = 0; kb < K; kb += GK) {
#pragma unroll
    for (int r = 0; r < (GK * GT) / GNT; ++r) {
      const int e = threadIdx.x + r * GNT;
      int kk, col;
      if (!trans) { kk = e / GT; col = e % GT; } else { col = e / GK; kk = e % GK; }
      const int64_t k = kb + kk;
      const int p = p0 + col, q = q0 + col;
      double vp = 0.0, vq = 0.0;
      if (k < K) {
        if (p < n) vp = trans ? src[p * lda + k] : src[k * lda + p];
        if (q < n) vq = trans ? src[q * lda + k] : src[k * lda + q];
      }
      P[kk][col] = vp;
      Q[kk][col] = vq;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const double b = Q[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += P[kk][ty + 8 * u] * b;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int p = p0 + ty + 8 * u, q = q0 + tx;
    if (p < n && q < n) G[static_cast<int64_t>(p) * n + q] = acc[u];
  }
}

// ------------------------------------------------------------------------------------
// Cholesky factorisations, one CTA per instance.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(CNT) kb_cholesky(const BInst* __restrict__ tab, int step,
                                                   int init_k, int which, unsigned* err,
                                                   int smem_bytes, int mixed, int ls_mode) {
  extern __shared__ double smem[];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, which != 0);
  if (!cu.active) return;
  const double eps = 2.220446049250313e-16, eps32 = 1.1920928955078125e-07;
  const bool tall = cu.I >= cu.L;
  if (which == 0) {
    const int n = cu.L;
    const int64_t nn = static_cast<int64_t>(n) * n;
    double* A = (nn * 8 <= smem_bytes) ? smem : d.Lrow;
    if (mixed) {
      float* A32 = (nn * 4 <= smem_bytes) ? reinterpret_cast<float*>(smem)
                                          : reinterpret_cast<float*>(d.Lrow);
      cholesky_cta_mixed<float>(d.M, n, ls_mode, static_cast<double>(n) * eps,
                                static_cast<double>(n) * eps32, A32, A, d.Lrow, d.Lcol,
                                d.invdiag, d.keep, d.info, err, static_cast<float*>(d.limg),
                                d.mimg);
      return;
    }
    cholesky_cta(d.M, n, ls_mode, static_cast<double>(n) * eps, A, d.Lrow, d.Lcol, d.invdiag,
                 d.keep, d.info, err, static_cast<double*>(d.limg), nullptr, nullptr);
    return;
  }
  const double tol = static_cast<double>(cu.I > cu.L ? cu.I : cu.L) * eps;
  if (which == 1) {
    const int n = tall ? cu.L : static_cast<int>(cu.I);
    const int64_t nn = static_cast<int64_t>(n) * n;
    double* A = (nn * 8 <= smem_bytes) ? smem : d.L1row;
    if (mixed && tall) {   // double-float first; a wide pass-1 factor feeds pass 2 (FP64)
      const double eps_ff = 9.094947017729282e-13;   // 2^-40
      float* Aff = (panel_floats<FFOps>(n) * 4 <= smem_bytes) ? reinterpret_cast<float*>(smem)
                                                               : nullptr;
      cholesky_cta_lev_mixed(d.G1, n, tol, tol / eps * eps_ff, Aff, A, d.L1row, d.L1col, d.inv1,
                             d.keep1, d.info1, err, d.img1);
      return;
    }
    cholesky_cta(d.G1, n, 1, tol, A, d.L1row, d.L1col, d.inv1, d.keep1, d.info1, err, d.img1,
                 nullptr, nullptr);
    return;
  }
  if (tall) return;
  const int n = static_cast<int>(cu.I);
  double* A = (static_cast<int64_t>(n) * n * 8 <= smem_bytes) ? smem : d.L2row;
  cholesky_cta(d.G2, n, 1, tol, A, d.L2row, d.L2col, d.inv2, d.keep2, d.info2, err, d.img2,
               nullptr, nullptr);
}

// The FP64 image of a double-float leverage factor from the FP32 planes the factorisation
// left in L1row / L1col (*info1 == 2; tall mixed instances only).
__global__ void __launch_bounds__(256) kb_ff_image(const BInst* __restrict__ tab, int step,
                                                   int init_k) {
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, true);
  if (!cu.active || cu.I < cu.L || *d.info1 != 2) return;
  const int n = cu.L;
  const int64_t count = static_cast<int64_t>(n) * (n + 1);
  const float* hi = reinterpret_cast<const float*>(d.L1row);
  const float* lo = reinterpret_cast<const float*>(d.L1col);
  for (int64_t e = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.y) * blockDim.x)
    d.img1[e] = static_cast<double>(hi[e]) + static_cast<double>(lo[e]);
}

// ------------------------------------------------------------------------------------
// Triangular solves: the LS solve (mode 2 mixed / mode 1 FP64) writing the new core, and
// the leverage rows with the fused p / CDF step.
// ------------------------------------------------------------------------------------
// Runtime choice of the register rows (QN = ceil(n/32)) and of shared-memory staging:
// n <= 128 always fits padded; beyond that the packed layout when it fits (`packed`), else
// the image stays in global memory.
template <typename T, int NB>
__device__ __forceinline__ void trsm_dispatch(bool smem, bool packed, unsigned char* sm,
                                              int64_t cta, int n,
                                              const double* Lrow, const double* Lcol,
                                              const double* invdiag, const int* info,
                                              int64_t nvec, const double* rhs, int64_t ld,
                                              int mode, const double* M, const T* Limg,
                                              const float* Mimg, int Rl, int Rr,
                                              double* core_out, double* ell,
                                              const CdfEpilogue& ep, int nctas) {
#define TB_ARGS sm, cta, n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, Rl, Rr, \
                core_out, ell, ep, nctas
  switch ((n + 31) / 32) {
    case 1: trsm_cta<T, 1, NB, true>(TB_ARGS); break;
    case 2: trsm_cta<T, 2, NB, true>(TB_ARGS); break;
    case 3: trsm_cta<T, 3, NB, true>(TB_ARGS); break;
    case 4: trsm_cta<T, 4, NB, true>(TB_ARGS); break;
    case 5:
      if (smem) trsm_cta<T, 5, NB, true>(TB_ARGS);
      else if (packed) trsm_cta<T, 5, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 5, NB, false>(TB_ARGS);
      break;
    case 6:
      if (packed) trsm_cta<T, 6, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 6, NB, false>(TB_ARGS);
      break;
    case 7:
      if (packed) trsm_cta<T, 7, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 7, NB, false>(TB_ARGS);
      break;
    case 8:
      if (packed) trsm_cta<T, 8, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 8, NB, false>(TB_ARGS);
      break;
    default: break;
  }
#undef TB_ARGS
}

template <typename T, int NB>
__global__ void __launch_bounds__(TW * 32) kb_solve(const BInst* __restrict__ tab, int step,
                                                    int smem_bytes) {
  extern __shared__ __align__(16) unsigned char sm[];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, 0, false);
  if (!cu.active) return;
  const int n = cu.L;
  const int64_t per = static_cast<int64_t>(TW) * NB;
  const int nctas = static_cast<int>((cu.I + per - 1) / per);
  if (static_cast<int>(blockIdx.y) >= nctas) return;
  const int mode = sizeof(T) == 4 ? 2 : 1;
  const CdfEpilogue none{};
  const bool smem = staged_bytes<T>(n, mode) <= static_cast<size_t>(smem_bytes);
  const bool packed = !smem && packed_bytes<T>(n) <= static_cast<size_t>(smem_bytes);
  trsm_dispatch<T, NB>(smem, packed, sm, blockIdx.y, n, d.Lrow, d.Lcol, d.invdiag, d.info, cu.I,
                       d.BT, n,
                       mode, d.M, static_cast<const T*>(d.limg), d.mimg, cu.Rl, cu.Rr,
                       d.cores[cu.n], nullptr, none, nctas);
}

__global__ void __launch_bounds__(TW * 32) kb_rows(const BInst* __restrict__ tab, int step,
                                                   int init_k, unsigned* err, int smem_bytes) {
  extern __shared__ __align__(16) unsigned char sm[];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, true);
  if (!cu.active) return;
  const bool tall = cu.I >= cu.L;
  const int n = tall ? cu.L : static_cast<int>(cu.I);
  const double* rhs = tall ? (cu.init ? d.cores[cu.n] : d.BT) : d.L1row;
  const int64_t ld = tall ? cu.L : cu.I;
  const double* Lr = tall ? d.L1row : d.L2row;
  const double* Lc = tall ? d.L1col : d.L2col;
  const double* iv = tall ? d.inv1 : d.inv2;
  const double* im = tall ? d.img1 : d.img2;
  const int nctas = static_cast<int>((cu.I + TW - 1) / TW);
  if (static_cast<int>(blockIdx.y) >= nctas) return;
  const CdfEpilogue ep{d.counter, d.p[cu.n], d.cdf[cu.n], cu.init ? nullptr : d.info, err};
  const bool smem = staged_bytes<double>(n, 0) <= static_cast<size_t>(smem_bytes);
  const bool packed = !smem && packed_bytes<double>(n) <= static_cast<size_t>(smem_bytes);
  trsm_dispatch<double, 1>(smem, packed, sm, blockIdx.y, n, Lr, Lc, iv, nullptr, cu.I, rhs, ld, 0,
                           nullptr,
                           im, nullptr, 1, 1, nullptr, d.ell, ep, nctas);
}

// ------------------------------------------------------------------------------------
// Serving: relative fit 1 - ||TR - X|| / ||X|| (Sec. 5.1) of every slot that completed a
// sweep in this tick, as kFitParts (or fewer) partial sums in a fixed order, then the stop
// rule (|fit_s - fit_{s-1}| < tol after two or more sweeps, or the sweep cap) and the step
// counters.
// ------------------------------------------------------------------------------------
// The slot's step is the last update of a sweep.
__device__ __forceinline__ bool fit_due(const BInst& d) {
  if (!d.slot) return false;
  const SlotState& s = *d.slot;
  return s.status == kSlotRunning && s.step >= 0 && s.step % d.N == d.N - 1;
}

// Partial sums of one slot's fit: one per CTA, at most kFitParts.
__device__ __forceinline__ int fit_parts(const FitSplit& f, bool xf64) {
  const int64_t nblk = fit_row_blocks(f, xf64);
  return nblk < kFitParts ? static_cast<int>(nblk) : kFitParts;
}

__device__ __forceinline__ void fit_args(const BInst& d, FitArgs& fa) {
  fa.N = d.N;
  for (int m = 0; m < d.N; ++m) {
    fa.core[m] = d.cores[m];
    fa.dims[m] = d.dims[m];
    fa.ranks[m] = d.ranks[m];
  }
}

constexpr int kFitRightCtas = 64;   // CTAs per slot forming the right factors

// Right factors of the fit: e-major W^T for the SIMT contraction, or the swizzled hi/lo
// tiles of the tensor-core contraction.
template <typename T>
__global__ void __launch_bounds__(FNT) kb_fit_right(const BInst* __restrict__ tab) {
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  __shared__ FitArgs fa;
  const BInst& d = tab[blockIdx.x];
  if (!fit_due(d)) return;
  if (threadIdx.x == 0) fit_args(d, fa);
  __syncthreads();
  const FitSplit f = fit_split(fa.N, fa.dims, fa.ranks);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t step = static_cast<int64_t>(gridDim.y) * (FNT / 32);
  const int64_t q0 = static_cast<int64_t>(blockIdx.y) * (FNT / 32) + warp;
  if constexpr (sizeof(T) == 4) {
    if (fit_use_tc(f, false)) {
      unsigned char* WS = static_cast<unsigned char*>(d.fitw);
      const int64_t ncol = (f.cols + FTN - 1) / FTN * FTN;
      for (int64_t q = q0; q < ncol; q += step)
        fit_right_tc_warp(fa, f, q, WS, chain[warp], slice[warp], lane);
      return;
    }
  }
  T* WT = static_cast<T*>(d.fitw);
  for (int64_t q = q0; q < f.cols; q += step)
    fit_right_warp<T>(fa, f, q, WT, chain[warp], slice[warp], lane);
}

// Slots whose contraction length K lies in (k_lo, k_hi] (two launches with different
// shared-memory sizes keep the common small-K case at several CTAs per SM).
template <typename T>
__global__ void __launch_bounds__(FNT) kb_fit(const BInst* __restrict__ tab, int k_lo, int k_hi) {
  extern __shared__ __align__(16) unsigned char fit_dyn[];
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  __shared__ double red[2 * (FNT / 32)];
  __shared__ FitArgs fa;
  const BInst& d = tab[blockIdx.x];
  if (!fit_due(d)) return;
  if (threadIdx.x == 0) fit_args(d, fa);
  __syncthreads();
  const FitSplit f = fit_split(fa.N, fa.dims, fa.ranks);
  if (fit_use_tc(f, sizeof(T) == 8) || f.K <= k_lo || f.K > k_hi) return;
  const int parts = fit_parts(f, sizeof(T) == 8);
  if (static_cast<int>(blockIdx.y) >= parts) return;
  double se = 0.0, sx = 0.0;
  fit_blocks<T>(fa, f, static_cast<const T*>(d.X), static_cast<const T*>(d.fitw), blockIdx.y,
                parts, fit_dyn, chain, slice, se, sx);
  fit_block_reduce(se, sx, red);
  if (threadIdx.x == 0) {
    d.fitp[blockIdx.y] = se;
    d.fitp[kFitParts + blockIdx.y] = sx;
  }
}

// Slots with FP32 X and K <= 128: the contraction on the tensor cores (fit_tc.cuh).
__global__ void __launch_bounds__(FNT, 1) kb_fit_tc(const BInst* __restrict__ tab,
                                                    unsigned* err) {
  extern __shared__ __align__(1024) unsigned char fit_tc_dyn[];
  __shared__ float chain[8][kMaxL];
  __shared__ float slice[8][kMaxL];
  __shared__ double red[2 * (FNT / 32)];
  __shared__ FitArgs fa;
  __shared__ FitTcShared sh;
  const BInst& d = tab[blockIdx.x];
  if (!fit_due(d) || d.xf64) return;
  if (threadIdx.x == 0) fit_args(d, fa);
  __syncthreads();
  const FitSplit f = fit_split(fa.N, fa.dims, fa.ranks);
  if (!fit_use_tc(f, false)) return;
  const int parts = fit_parts(f, false);
  if (static_cast<int>(blockIdx.y) >= parts) return;
  double se = 0.0, sx = 0.0;
  fit_tc_blocks(fa, f, static_cast<const float*>(d.X),
                static_cast<const unsigned char*>(d.fitw),
                blockIdx.y, parts, fit_tc_dyn, chain, slice, sh, err, se, sx);
  fit_block_reduce(se, sx, red);
  if (threadIdx.x == 0) {
    d.fitp[blockIdx.y] = se;
    d.fitp[kFitParts + blockIdx.y] = sx;
  }
}

__global__ void __launch_bounds__(128) kb_advance(const BInst* __restrict__ tab, int count,
                                                  int xf64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const BInst& d = tab[i];
  if (!d.slot) return;
  SlotState& s = *d.slot;
  if (s.status != kSlotRunning) return;
  const int t = s.step;
  if (t >= 0 && *d.info != 0) s.singular += 1;
  if (fit_due(d)) {
    const FitSplit f = fit_split(d.N, d.dims, d.ranks);
    const int parts = fit_parts(f, xf64 != 0);
    double se = 0.0, sx = 0.0;
    for (int q = 0; q < parts; ++q) {
      se += d.fitp[q];
      sx += d.fitp[kFitParts + q];
    }
    const double rel = sx > 0.0 ? sqrt(se / sx) : (se > 0.0 ? INFINITY : 0.0);
    const double fit = 1.0 - rel;
    const int sw = s.sweeps + 1;
    s.sweeps = sw;
    s.fit_prev = s.fit;
    s.fit = fit;
    if (sw <= kMaxServedSweeps) d.hist[sw - 1] = fit;
    if (!isfinite(fit)) s.status = kSlotFailed;
    else if (sw >= 2 && fabs(fit - s.fit_prev) < s.tol) s.status = kSlotConverged;
    else if (sw >= s.max_sweeps) s.status = kSlotCapped;
  }
  s.step = t + 1;
}

constexpr int kDyn = 200 * 1024;

int smem_for_cholesky(int nmax) {
  const int64_t need = static_cast<int64_t>(nmax) * nmax * 8;
  const int64_t ff = panel_floats<FFOps>(nmax) * 4;
  if ((ff > need ? ff : need) <= kDyn) return static_cast<int>(ff > need ? ff : need);
  return need <= kDyn ? static_cast<int>(need) : 0;
}

}  // namespace

cudaError_t bl_init_cores(const BLaunch& b, cudaStream_t st) {
  dim3 grid(b.count, 16);
  kb_init_cores<<<grid, 256, 0, st>>>(b.tab);
  return cudaGetLastError();
}

cudaError_t bl_sample_chain_gather(const BLaunch& b, int step, cudaStream_t st) {
  const int spw = b.spw >= 1 && b.spw <= kSpwMax ? b.spw : 4;
  const int64_t per = SW * spw;
  dim3 grid(b.count, static_cast<unsigned>((b.Jmax + per - 1) / per));
  if (b.f64 && b.xf64) kb_sample<double, double><<<grid, SW * 32, 0, st>>>(b.tab, step, spw);
  else if (b.f64) kb_sample<double, float><<<grid, SW * 32, 0, st>>>(b.tab, step, spw);
  else if (b.xf64) kb_sample<float, double><<<grid, SW * 32, 0, st>>>(b.tab, step, spw);
  else kb_sample<float, float><<<grid, SW * 32, 0, st>>>(b.tab, step, spw);
  return cudaGetLastError();
}

template <int TILE>
cudaError_t contract_tile(const BLaunch& b, int step, cudaStream_t st) {
  const int ntr = (b.Lmax + TILE - 1) / TILE;
  const int64_t ntc = (b.Lmax + b.Imax + TILE - 1) / TILE;
  dim3 grid(b.count, static_cast<unsigned>(ntr * ntc));
  constexpr int CT = (TILE / 4) * (TILE / 4);
  if (b.f64) kb_contract<double, TILE><<<grid, CT, 0, st>>>(b.tab, step);
  else kb_contract<float, TILE><<<grid, CT, 0, st>>>(b.tab, step);
  return cudaGetLastError();
}

cudaError_t bl_contract(const BLaunch& b, int step, cudaStream_t st) {
  return b.ctile == 32 ? contract_tile<32>(b, step, st) : contract_tile<64>(b, step, st);
}

cudaError_t bl_cholesky(const BLaunch& b, int step, int init_k, int which, unsigned* err,
                        cudaStream_t st) {
  const int nmax = which == 0 ? b.Lmax : (which == 1 ? b.n1max : b.n2max);
  if (nmax <= 0) return cudaSuccess;
  const int dyn = smem_for_cholesky(nmax);
  kb_cholesky<<<b.count, CNT, dyn, st>>>(b.tab, step, init_k, which, err, dyn, b.f64 ? 0 : 1,
                                          b.ls_mode);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || which != 1 || b.f64) return e;
  // double-float leverage factors leave FP32 planes: their FP64 image
  const int64_t count = static_cast<int64_t>(nmax) * (nmax + 1);
  dim3 grid(b.count, static_cast<unsigned>((count + 255) / 256 < 16 ? (count + 255) / 256 : 16));
  kb_ff_image<<<grid, 256, 0, st>>>(b.tab, step, init_k);
  return cudaGetLastError();
}

// Dynamic shared memory for the solve kernels: enough for every instance that takes the
// shared-memory path (every n <= 128 does; n >= 161 never does).
template <typename T>
int solve_smem(int nmax, int mode) {
  const int n = nmax < 160 ? nmax : 160;
  size_t need = staged_bytes<T>(n, mode);
  const size_t pk = packed_bytes<T>(nmax);
  if (nmax > 128 && pk <= static_cast<size_t>(kDyn) && pk > need) need = pk;
  return need <= static_cast<size_t>(kDyn) ? static_cast<int>(need) : kDyn;
}

cudaError_t bl_solve(const BLaunch& b, int step, cudaStream_t st) {
  if (b.f64) {
    const int dyn = solve_smem<double>(b.Lmax, 1);
    dim3 grid(b.count, static_cast<unsigned>((b.Imax + TW - 1) / TW));
    kb_solve<double, 1><<<grid, TW * 32, dyn, st>>>(b.tab, step, dyn);
  } else {
    const int dyn = solve_smem<float>(b.Lmax, 2);
    dim3 grid(b.count, static_cast<unsigned>((b.Imax + 2 * TW - 1) / (2 * TW)));
    kb_solve<float, 2><<<grid, TW * 32, dyn, st>>>(b.tab, step, dyn);
  }
  return cudaGetLastError();
}

cudaError_t bl_gram(const BLaunch& b, int step, int init_k, int pass, cudaStream_t st) {
  const int nmax = pass == 1 ? b.n1max : b.n2max;
  if (nmax <= 0) return cudaSuccess;
  const int nt = (nmax + GT - 1) / GT;
  dim3 grid(b.count, nt * nt);
  kb_gram<<<grid, GNT, 0, st>>>(b.tab, step, init_k, pass);
  return cudaGetLastError();
}

cudaError_t bl_leverage_rows(const BLaunch& b, int step, int init_k, unsigned* err,
                             cudaStream_t st) {
  const int nmax = b.n1max > b.n2max ? b.n1max : b.n2max;
  const int dyn = solve_smem<double>(nmax, 0);
  dim3 grid(b.count, static_cast<unsigned>((b.Imax + TW - 1) / TW));
  kb_rows<<<grid, TW * 32, dyn, st>>>(b.tab, step, init_k, err, dyn);
  return cudaGetLastError();
}

cudaError_t bl_fit(const BLaunch& b, unsigned* err, cudaStream_t st) {
  dim3 rgrid(b.count, kFitRightCtas);
  dim3 grid(b.count, kFitParts);
  constexpr int kSplitK = 128;
  const int k_small = b.Lmax < kSplitK ? b.Lmax : kSplitK;
  if (b.xf64) {
    kb_fit_right<double><<<rgrid, FNT, 0, st>>>(b.tab);
    kb_fit<double><<<grid, FNT, fit_smem_bytes<double>(k_small), st>>>(b.tab, 0, kSplitK);
    if (b.Lmax > kSplitK)
      kb_fit<double><<<grid, FNT, fit_smem_bytes<double>(b.Lmax), st>>>(b.tab, kSplitK, kMaxL);
  } else {
    kb_fit_right<float><<<rgrid, FNT, 0, st>>>(b.tab);
    kb_fit_tc<<<grid, FNT, kFitTcSmem, st>>>(b.tab, err);
    if (b.Lmax > kFitTcMaxK)
      kb_fit<float><<<grid, FNT, fit_smem_bytes<float>(b.Lmax), st>>>(b.tab, kFitTcMaxK, kMaxL);
  }
  return cudaGetLastError();
}

cudaError_t bl_advance(const BLaunch& b, cudaStream_t st) {
  kb_advance<<<(b.count + 127) / 128, 128, 0, st>>>(b.tab, b.count, b.xf64 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t batched_attributes() {
  cudaError_t e = cudaFuncSetAttribute(kb_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kDyn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kb_solve<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kb_solve<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kb_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kb_fit<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(fit_smem_bytes<float>(kMaxL)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kb_fit_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kFitTcSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kb_fit<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(fit_smem_bytes<double>(kMaxL)));
}

}  // namespace trk
