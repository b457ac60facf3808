// FP64 dense kernels of the hot path:
//   * Gram matrices and the Cholesky-based thin QR behind the leverage scores of a core
//     (row a1: Def. 3.3 and eq. for p^(n)); R of the thin QR of A is the Cholesky factor
//     of A^T A, and Q = A R^-1, so ell_i = || R^-T a_i ||^2.
//   * fixed-order reduction of split partials;
//   * Cholesky factorisation of the normal matrix, the triangular solves for all I_n
//     right-hand sides and one step of iterative refinement (row a6);
//   * p = ell / sum(ell) and its prefix sum (the CDF used by the sampler).
#include <float.h>

#include "common.cuh"

namespace trk {
namespace {

// ------------------------------------------------------------------------------------
// Gram: partial[s][p][q] = sum_{t in chunk s} X(t, p) X(t, q), tiles with tp <= tq only.
// X(t, p) = A[t*lda + p] (trans = false) or A[p*lda + t] (trans = true).
// ------------------------------------------------------------------------------------
constexpr int GT = 32, GK = 32, GNT = 256;

__global__ void __launch_bounds__(GNT) k_gram(const double* __restrict__ A, int64_t K, int n,
                                              int64_t lda, bool trans, int64_t chunk,
                                              double* __restrict__ partial) {
  __shared__ double P[GK][GT + 1];
  __shared__ double Q[GK][GT + 1];
  const int nt = (n + GT - 1) / GT;
  int tp = 0, rem = blockIdx.x;
  while (rem >= nt - tp) { rem -= nt - tp; ++tp; }
  const int tq = tp + rem;
  const int p0 = tp * GT, q0 = tq * GT;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t k1 = (k0 + chunk < K) ? k0 + chunk : K;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  double acc[4] = {0, 0, 0, 0};
  for (int64_t kb = k0; kb < k1; kb += GK) {
#pragma unroll
    for (int r = 0; r < (GK * GT) / GNT; ++r) {
      const int e = threadIdx.x + r * GNT;
      int kk, col;
      if (!trans) { kk = e / GT; col = e % GT; } else { col = e / GK; kk = e % GK; }
      const int64_t t = kb + kk;
      const int p = p0 + col, q = q0 + col;
      double vp = 0.0, vq = 0.0;
      if (t < k1) {
        if (p < n) vp = trans ? A[p * lda + t] : A[t * lda + p];
        if (q < n) vq = trans ? A[q * lda + t] : A[t * lda + q];
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
  double* out = partial + static_cast<int64_t>(blockIdx.y) * n * n;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int p = p0 + ty + 8 * u, q = q0 + tx;
    if (p < n && q < n) out[static_cast<int64_t>(p) * n + q] = acc[u];
  }
}

// ------------------------------------------------------------------------------------
// Fixed-order reduction of split partials into an FP64 block (optionally transposed).
// ------------------------------------------------------------------------------------
template <typename TP>
__global__ void __launch_bounds__(256) k_reduce(const TP* __restrict__ partial, int splits,
                                                int64_t pstride, int64_t pld, int64_t row0,
                                                int64_t nrows, int64_t col0, int64_t ncols,
                                                double* __restrict__ out, int64_t ldo,
                                                bool transpose) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 32;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t r = r0 + ty + 8 * u, c = c0 + tx;
    double s = 0.0;
    if (r < nrows && c < ncols) {
      const TP* src = partial + (row0 + r) * pld + col0 + c;
      for (int q = 0; q < splits; ++q) s += static_cast<double>(src[q * pstride]);
    }
    tile[ty + 8 * u][tx] = s;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (!transpose) {
      const int64_t r = r0 + ty + 8 * u, c = c0 + tx;
      if (r < nrows && c < ncols) out[r * ldo + c] = tile[ty + 8 * u][tx];
    } else {
      const int64_t c = c0 + ty + 8 * u, r = r0 + tx;  // out[c][r]
      if (r < nrows && c < ncols) out[c * ldo + r] = tile[tx][ty + 8 * u];
    }
  }
}

// ------------------------------------------------------------------------------------
// Right-looking Cholesky in one CTA (shared memory when it fits, else in place in Lrow).
// ------------------------------------------------------------------------------------
constexpr int CNT = 512;

__global__ void __launch_bounds__(CNT) k_cholesky(const double* __restrict__ G, int n, int mode,
                                                  double tol_scale, double* Lrow, double* Lcol,
                                                  double* invdiag, int* keep_out, int* info,
                                                  unsigned* err, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double colk[kMaxL];
  __shared__ int keepv[kMaxL];
  __shared__ double s_piv, s_tol;
  __shared__ int s_keep, s_stop;
  double* A = use_smem ? smem : Lrow;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = CNT / 32;
  for (int e = tid; e < n * n; e += CNT) {
    const int i = e / n, j = e - (e / n) * n;
    A[e] = (j <= i) ? G[static_cast<int64_t>(j) * n + i] : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double md = 0.0;
    for (int i = 0; i < n; ++i) md = fmax(md, A[i * n + i]);
    s_tol = tol_scale * md;
    s_stop = 0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double d = A[k * n + k];
      const bool ok = d > s_tol;          // false for NaN and for an all-zero matrix
      s_keep = ok ? 1 : 0;
      s_piv = ok ? sqrt(d) : 0.0;
      if (!ok && mode == 0) s_stop = k + 1;
      keepv[k] = s_keep;
    }
    __syncthreads();
    if (s_stop) break;
    const bool kp = s_keep != 0;
    const double piv = s_piv;
    for (int i = k + tid; i < n; i += CNT) {
      double v;
      if (!kp) v = 0.0;
      else v = (i == k) ? piv : A[i * n + k] / piv;
      A[i * n + k] = v;
      colk[i] = v;
    }
    __syncthreads();
    if (kp) {
      const int m = n - k - 1;
      for (int ii = warp; ii < m; ii += nw) {
        const int i = k + 1 + ii;
        const double li = colk[i];
        for (int jj = lane; jj <= ii; jj += 32) A[i * n + k + 1 + jj] -= li * colk[k + 1 + jj];
      }
    }
    __syncthreads();
  }
  __syncthreads();
  const int stop = s_stop;
  if (tid == 0) {
    *info = stop;
    if (stop) atomicOr(err, kErrSingular);
  }
  if (stop) return;
  for (int e = tid; e < n * n; e += CNT) {
    const int i = e / n, j = e - (e / n) * n;
    const double v = (j <= i) ? A[e] : 0.0;
    Lrow[e] = v;
    Lcol[static_cast<int64_t>(j) * n + i] = v;
  }
  for (int k = tid; k < n; k += CNT) {
    keep_out[k] = keepv[k];
    invdiag[k] = keepv[k] ? 1.0 / A[k * n + k] : 0.0;
  }
}

// In-place solve of L y = x (forward) by one warp; x in shared memory, Lcol = L^T.
__device__ __forceinline__ void warp_forward(double* x, int n, const double* __restrict__ Lcol,
                                             const double* __restrict__ invdiag, int lane) {
  for (int c = 0; c < n; ++c) {
    __syncwarp();
    const double xc = x[c] * invdiag[c];
    __syncwarp();
    const double* col = Lcol + static_cast<int64_t>(c) * n;
    for (int r = c + 1 + lane; r < n; r += 32) x[r] -= col[r] * xc;
    if (lane == 0) x[c] = xc;
  }
  __syncwarp();
}

// In-place solve of L^T z = y (backward) by one warp; Lrow row c = column c of L^T.
__device__ __forceinline__ void warp_backward(double* x, int n, const double* __restrict__ Lrow,
                                              const double* __restrict__ invdiag, int lane) {
  for (int c = n - 1; c >= 0; --c) {
    __syncwarp();
    const double zc = x[c] * invdiag[c];
    __syncwarp();
    const double* row = Lrow + static_cast<int64_t>(c) * n;
    for (int r = lane; r < c; r += 32) x[r] -= row[r] * zc;
    if (lane == 0) x[c] = zc;
  }
  __syncwarp();
}

constexpr int SW = 4;  // warps per CTA in the RHS kernel

__global__ void __launch_bounds__(SW * 32) k_solve_rhs(const double* __restrict__ BT,
                                                       const double* __restrict__ M, int L,
                                                       int Rl, int Rr, int64_t I,
                                                       const double* __restrict__ Lrow,
                                                       const double* __restrict__ Lcol,
                                                       const double* __restrict__ invdiag,
                                                       bool refine, const int* __restrict__ info,
                                                       double* __restrict__ core_out) {
  __shared__ double sx[SW][kMaxL];
  __shared__ double sb[SW][kMaxL];
  if (*info != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * SW + warp;
  if (i >= I) return;
  double* x = sx[warp];
  double* b = sb[warp];
  for (int c = lane; c < L; c += 32) { const double v = BT[i * L + c]; b[c] = v; x[c] = v; }
  warp_forward(x, L, Lcol, invdiag, lane);
  warp_backward(x, L, Lrow, invdiag, lane);
  if (refine) {
    // r = b - M z (M symmetric: row t of M gives column t), then z += M^-1 r.
    double acc[kMaxL / 32];
#pragma unroll
    for (int q = 0; q < kMaxL / 32; ++q) acc[q] = 0.0;
    for (int t = 0; t < L; ++t) {
      const double zt = x[t];
      const double* row = M + static_cast<int64_t>(t) * L;
#pragma unroll
      for (int q = 0; q < kMaxL / 32; ++q) {
        const int c = lane + 32 * q;
        if (c < L) acc[q] += row[c] * zt;
      }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kMaxL / 32; ++q) {
      const int c = lane + 32 * q;
      if (c < L) b[c] = b[c] - acc[q];
    }
    warp_forward(b, L, Lcol, invdiag, lane);
    warp_backward(b, L, Lrow, invdiag, lane);
    for (int c = lane; c < L; c += 32) x[c] += b[c];
    __syncwarp();
  }
  double* out = core_out + i * L;
  for (int c = lane; c < L; c += 32) {
    const int a = c % Rl, bb = c / Rl;
    out[a * Rr + bb] = x[c];
  }
}

constexpr int LW = 8;  // warps per CTA in the leverage-row kernel

__global__ void __launch_bounds__(LW * 32) k_leverage_rows(const double* __restrict__ A,
                                                           int64_t rows, int n, int64_t lda,
                                                           const double* __restrict__ Lcol,
                                                           const double* __restrict__ invdiag,
                                                           double* __restrict__ ell) {
  __shared__ double sx[LW][kMaxL];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * LW + warp;
  if (i >= rows) return;
  double* x = sx[warp];
  for (int c = lane; c < n; c += 32) x[c] = A[i * lda + c];
  warp_forward(x, n, Lcol, invdiag, lane);
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += x[c] * x[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) ell[i] = s;
}

constexpr int PNT = 1024;

__global__ void __launch_bounds__(PNT) k_cdf(const double* __restrict__ ell, int64_t I,
                                             double* __restrict__ p, double* __restrict__ cdf,
                                             unsigned* err) {
  __shared__ double part[PNT];
  __shared__ double s_total;
  const int t = threadIdx.x;
  const int64_t chunk = (I + PNT - 1) / PNT;
  const int64_t b = t * chunk, e = (b + chunk < I) ? b + chunk : I;
  double s = 0.0;
  for (int64_t i = b; i < e; ++i) s += ell[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
    for (int q = 0; q < PNT; ++q) tot += part[q];
    s_total = tot;
  }
  __syncthreads();
  const double total = s_total;
  const bool bad = !(total > 0.0) || !isfinite(total);
  if (bad) {
    for (int64_t i = b; i < e; ++i) {
      p[i] = 1.0 / static_cast<double>(I);
      cdf[i] = static_cast<double>(i + 1) / static_cast<double>(I);
    }
    if (t == 0) atomicOr(err, kErrSingular);
    return;
  }
  s = 0.0;
  for (int64_t i = b; i < e; ++i) s += ell[i] / total;
  __syncthreads();
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    double run = 0.0;
    for (int q = 0; q < PNT; ++q) { const double v = part[q]; part[q] = run; run += v; }
  }
  __syncthreads();
  double run = part[t];
  for (int64_t i = b; i < e; ++i) {
    const double pi = ell[i] / total;
    p[i] = pi;
    run += pi;
    cdf[i] = run;
  }
}

// ------------------------------------------------------------------------------------
// N(0,1) by Philox4x32-10 + Box-Muller (Box & Muller, 1958): pair q uses counter
// (q lo, q hi, stream_id, 0x4E4F524D), two 53-bit uniforms u1, u2; r = sqrt(-2 ln(1-u1)),
// (r cos 2 pi u2, r sin 2 pi u2).
// ------------------------------------------------------------------------------------
__global__ void k_init_normal(double* __restrict__ out, int64_t count, uint32_t k0, uint32_t k1,
                              uint32_t stream_id) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (2 * q >= count) return;
  const u32x4 r = philox4x32_10(u32x4{static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                      stream_id, 0x4E4F524Du},
                                k0, k1);
  const double u1 = u53(r.x, r.y), u2 = u53(r.z, r.w);
  const double rad = sqrt(-2.0 * log1p(-u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  out[2 * q] = rad * c;
  if (2 * q + 1 < count) out[2 * q + 1] = rad * s;
}

int plan_splits(int64_t K, int tiles, int min_chunk, int64_t* chunk) {
  int64_t s = (2 * 152 + tiles - 1) / tiles;
  const int64_t maxs = (K + min_chunk - 1) / min_chunk;
  if (s > maxs) s = maxs;
  if (s < 1) s = 1;
  int64_t c = (K + s - 1) / s;
  c = (c + GK - 1) / GK * GK;
  s = (K + c - 1) / c;
  if (s < 1) s = 1;
  *chunk = c;
  return static_cast<int>(s);
}

}  // namespace

size_t gram_workspace(int64_t rows, int cols, bool trans, int* splits) {
  const int64_t K = trans ? cols : rows;
  const int n = trans ? static_cast<int>(rows) : cols;
  const int nt = (n + GT - 1) / GT;
  int64_t chunk;
  *splits = plan_splits(K, nt * (nt + 1) / 2, GK, &chunk);
  return static_cast<size_t>(*splits) * n * n * sizeof(double);
}

cudaError_t launch_gram(const double* A, int64_t rows, int cols, int64_t lda, bool trans,
                        double* partial, int splits, cudaStream_t st) {
  const int64_t K = trans ? cols : rows;
  const int n = trans ? static_cast<int>(rows) : cols;
  const int nt = (n + GT - 1) / GT;
  int64_t chunk;
  const int s = plan_splits(K, nt * (nt + 1) / 2, GK, &chunk);
  if (s != splits) return cudaErrorInvalidValue;
  dim3 grid(nt * (nt + 1) / 2, s);
  k_gram<<<grid, GNT, 0, st>>>(A, K, n, lda, trans, chunk, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const void* partial, bool partial_f32, int splits, int64_t pstride,
                          int64_t pld, int64_t row0, int64_t nrows, int64_t col0,
                          int64_t ncols, double* out, int64_t ldo, bool transpose,
                          cudaStream_t st) {
  if (nrows <= 0 || ncols <= 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>((ncols + 31) / 32), static_cast<unsigned>((nrows + 31) / 32));
  if (partial_f32)
    k_reduce<float><<<grid, 256, 0, st>>>(static_cast<const float*>(partial), splits, pstride,
                                          pld, row0, nrows, col0, ncols, out, ldo, transpose);
  else
    k_reduce<double><<<grid, 256, 0, st>>>(static_cast<const double*>(partial), splits,
                                           pstride, pld, row0, nrows, col0, ncols, out, ldo,
                                           transpose);
  return cudaGetLastError();
}

cudaError_t launch_cholesky(const double* G, int n, int mode, double tol_scale, double* Lrow,
                            double* Lcol, double* invdiag, int* keep, int* info, unsigned* err,
                            cudaStream_t st) {
  const size_t bytes = static_cast<size_t>(n) * n * sizeof(double);
  const int use_smem = bytes <= 200 * 1024 ? 1 : 0;
  const size_t dyn = use_smem ? bytes : 0;
  if (use_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(dyn));
    if (e != cudaSuccess) return e;
  }
  k_cholesky<<<1, CNT, dyn, st>>>(G, n, mode, tol_scale, Lrow, Lcol, invdiag, keep, info, err,
                                  use_smem);
  return cudaGetLastError();
}

cudaError_t launch_solve_rhs(const double* BT, const double* M, int L, int Rl, int Rr,
                             int64_t I, const double* Lrow, const double* Lcol,
                             const double* invdiag, bool refine, const int* info,
                             double* core_out, cudaStream_t st) {
  if (I <= 0) return cudaSuccess;
  const int64_t blocks = (I + SW - 1) / SW;
  k_solve_rhs<<<static_cast<unsigned>(blocks), SW * 32, 0, st>>>(
      BT, M, L, Rl, Rr, I, Lrow, Lcol, invdiag, refine, info, core_out);
  return cudaGetLastError();
}

cudaError_t launch_leverage_rows(const double* A, int64_t rows, int n, int64_t lda,
                                 const double* Lcol, const double* invdiag, const int* keep,
                                 double* ell, cudaStream_t st) {
  (void)keep;  // dropped columns carry invdiag = 0, so they contribute nothing
  if (rows <= 0) return cudaSuccess;
  const int64_t blocks = (rows + LW - 1) / LW;
  k_leverage_rows<<<static_cast<unsigned>(blocks), LW * 32, 0, st>>>(A, rows, n, lda, Lcol,
                                                                      invdiag, ell);
  return cudaGetLastError();
}

cudaError_t launch_cdf(const double* ell, int64_t I, double* p, double* cdf, unsigned* err,
                       cudaStream_t st) {
  k_cdf<<<1, PNT, 0, st>>>(ell, I, p, cdf, err);
  return cudaGetLastError();
}

cudaError_t launch_init_normal(double* out, int64_t count, uint64_t seed, uint32_t stream_id,
                               cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t pairs = (count + 1) / 2;
  const int threads = 256;
  k_init_normal<<<static_cast<unsigned>((pairs + threads - 1) / threads), threads, 0, st>>>(
      out, count, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), stream_id);
  return cudaGetLastError();
}

}  // namespace trk
