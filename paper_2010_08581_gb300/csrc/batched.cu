// Batched stages of TR-ALS-Sampled (Alg. 2 per instance, Alg. 3 + Alg. 4 for the sketch):
// one launch per stage for every instance of the table; see batched.cuh. This file holds
// the initial cores, the draws with their rows and fibres, the normal-equation contraction
// and the leverage Grams; the factorisations, solves and fit live in batched_chol.cu,
// batched_solve32.cu, batched_solve64.cu and batched_fit.cu.
#include "batched_kern.cuh"
#include "draw.cuh"

namespace trk {
namespace {

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
//           (the core at initialisation and, under the column-dropping LS rule, after each
//           update; B^T during the updates otherwise);
//   pass 2 (wide modes only): G2 = C^T C (I x I), C = the pass-1 factor.
// ------------------------------------------------------------------------------------
constexpr int GT = 32, GK = 32, GNT = 256;

__global__ void __launch_bounds__(GNT) kb_gram(const BInst* __restrict__ tab, int step, int init_k,
                                               int pass, int from_core) {
  __shared__ double P[GK][GT + 1];
  __shared__ double Q[GK][GT + 1];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, true);
  if (!cu.active) return;
  const bool tall = cu.I >= cu.L;
  if (pass == 2 && tall) return;
  const double* S = (cu.init || from_core) ? d.cores[cu.n] : d.BT;
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

cudaError_t bl_gram(const BLaunch& b, int step, int init_k, int pass, cudaStream_t st) {
  const int nmax = pass == 1 ? b.n1max : b.n2max;
  if (nmax <= 0) return cudaSuccess;
  const int nt = (nmax + GT - 1) / GT;
  dim3 grid(b.count, nt * nt);
  kb_gram<<<grid, GNT, 0, st>>>(b.tab, step, init_k, pass, b.ls_mode == 1 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t bl_solve(const BLaunch& b, int step, cudaStream_t st) {
  return b.f64 ? bl_solve_f64(b, step, st) : bl_solve_f32(b, step, st);
}

cudaError_t batched_attributes() {
  cudaError_t e = batched_chol_attributes();
  if (e != cudaSuccess) return e;
  e = batched_solve32_attributes();
  if (e != cudaSuccess) return e;
  e = batched_solve64_attributes();
  if (e != cudaSuccess) return e;
  return batched_fit_attributes();
}

}  // namespace trk
