// One-CTA Cholesky factorisation G = L L^T (n <= 256), shared by the single-problem kernel
// and the batched kernel. Used for the normal matrix of the sampled LS (row a6, Alg. 2 LS
// step) and for the R factor of the Cholesky-based thin QR behind the leverage scores
// (row a1).
//
// Right-looking with one column of look-ahead. At step k column k is final; warp 0 applies
// column k's update to column k+1 only, takes its pivot (rsqrt) and scales it, while warps
// 1.. apply column k's rank-1 update to the trailing triangle of columns >= k+2. One barrier
// per column. A is the n x n work array (shared memory, or global scratch).
//
// The working type T is double or float. In FP64 the trailing triangle's (m+1)m/2 entries
// are spread evenly over the threads (every lane busy: the FP64 pipe is the bound); every
// update is one fused multiply-add, a_ij = fma(-l_ik, l_jk, a_ij), so that the cluster
// kernel (cholesky_cluster.cu), which applies the same updates in the same order, gives
// the same factor. In FP32 (the mixed-precision LS step, whose triangular solves already
// run in FP32) a warp takes whole rows and its lanes the columns, with no index arithmetic
// per entry.
//
// mode 0 (solve): a pivot <= tol_scale * max diag stops the factorisation (*info = column
// + 1, singular bit). mode 1 (leverage): such a column is dropped (zero, keep = 0).
// A non-final attempt (`final_attempt` false: the FP32 try of the mixed LS step) that stops
// writes nothing and returns false; its caller then factors in FP64.
// Besides L (row- and column-major, if Lrow/Lcol are given) the kernel can write padded
// images that the triangular-solve kernels copy straight into shared memory:
// img[c*(n+1) + r] = L[r][c] in FP64 and/or FP32, and the FP32 image of the symmetric input.
#pragma once

#include "common.cuh"

namespace trk {

constexpr int CNT = 512;

__device__ __forceinline__ double chol_rsqrt(double d) { return rsqrt(d); }
__device__ __forceinline__ float chol_rsqrt(float d) { return rsqrtf(d); }
__device__ __forceinline__ double chol_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float chol_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double chol_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float chol_max(float a, float b) { return fmaxf(a, b); }

template <typename T>
__device__ __forceinline__ bool cholesky_cta(const double* __restrict__ G, int n, int mode,
                                             double tol_scale, T* A, double* Lrow,
                                             double* Lcol, double* invdiag, int* keep_out,
                                             int* info, unsigned* err, double* img64,
                                             float* img32, float* gimg32,
                                             bool final_attempt = true) {
  __shared__ T colbuf[2][kMaxL];
  __shared__ int keepv[kMaxL];
  __shared__ T s_tol;
  __shared__ int s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = n + 1;
  for (int e = tid; e < n * n; e += CNT) {
    const int i = e / n, j = e - (e / n) * n;
    if (j <= i) {
      const double g = G[static_cast<int64_t>(j) * n + i];
      A[e] = static_cast<T>(g);
      if (gimg32) {
        gimg32[j * np + i] = static_cast<float>(g);
        gimg32[i * np + j] = static_cast<float>(g);
      }
    } else {
      A[e] = T(0);
    }
  }
  __syncthreads();
  if (warp == 0) {
    T md = T(0);
    for (int i = lane; i < n; i += 32) md = chol_max(md, A[i * n + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = chol_max(md, __shfl_xor_sync(0xffffffffu, md, o));
    const T tol = static_cast<T>(tol_scale) * md;
    const T d = A[0];
    const bool ok = d > tol;                  // false for NaN and non-positive pivots
    const T inv = ok ? chol_rsqrt(d) : T(0);
    for (int i = lane; i < n; i += 32) {
      const T v = ok ? ((i == 0) ? d * inv : A[i * n] * inv) : T(0);
      A[i * n] = v;
      colbuf[0][i] = v;
    }
    if (lane == 0) {
      s_tol = tol;
      keepv[0] = ok ? 1 : 0;
      s_stop = (!ok && mode == 0) ? 1 : 0;
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (s_stop) break;
    const T* cur = colbuf[k & 1];
    T* nxt = colbuf[(k + 1) & 1];
    const bool kp = keepv[k] != 0;
    if (warp == 0) {
      if (k + 1 < n) {
        // column k+1: a_i = A[i][k+1] - L[i][k] L[k+1][k]; pivot; scale
        const T lk1 = cur[k + 1];
        T a[kMaxL / 32];
#pragma unroll
        for (int q = 0; q < kMaxL / 32; ++q) {
          const int i = k + 1 + lane + 32 * q;
          a[q] = T(0);
          if (i < n) a[q] = kp ? chol_fma(-cur[i], lk1, A[i * n + k + 1]) : A[i * n + k + 1];
        }
        const T d = __shfl_sync(0xffffffffu, a[0], 0);   // row k+1: lane 0, q = 0
        const bool ok = d > s_tol;
        const T inv = ok ? chol_rsqrt(d) : T(0);
#pragma unroll
        for (int q = 0; q < kMaxL / 32; ++q) {
          const int i = k + 1 + lane + 32 * q;
          if (i < n) {
            const T v = ok ? ((i == k + 1) ? d * inv : a[q] * inv) : T(0);
            A[i * n + k + 1] = v;
            nxt[i] = v;
          }
        }
        if (lane == 0) {
          keepv[k + 1] = ok ? 1 : 0;
          if (!ok && mode == 0) s_stop = k + 2;
        }
      }
    } else if (!kp) {
      // a dropped column updates nothing
    } else if constexpr (sizeof(T) == 4) {
      // trailing triangle, FP32: warp w takes rows k+2+(w-1), k+2+(w-1)+(W-1), ...; its
      // lanes the columns k+2 .. i of the row
      const int j0 = k + 2;
      for (int i = j0 + warp - 1; i < n; i += CNT / 32 - 1) {
        const T li = cur[i];
        T* row = A + i * n;
        for (int j = j0 + lane; j <= i; j += 32) row[j] = chol_fma(-li, cur[j], row[j]);
      }
    } else {
      // trailing triangle of columns >= k+2: rows i >= j >= k+2
      const int m = n - k - 2;
      const int P = m > 0 ? m * (m + 1) / 2 : 0;
      for (int e = tid - 32; e < P; e += CNT - 32) {
        int ii = static_cast<int>((sqrtf(8.0f * static_cast<float>(e) + 1.0f) - 1.0f) * 0.5f);
        while (ii * (ii + 1) / 2 > e) --ii;
        while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
        const int jj = e - ii * (ii + 1) / 2;
        const int i = k + 2 + ii, j = k + 2 + jj;
        A[i * n + j] = fma(-cur[i], cur[j], A[i * n + j]);
      }
    }
    __syncthreads();
  }
  const int stop = s_stop;
  if (stop && !final_attempt) return false;
  if (tid == 0) {
    *info = stop;
    if (stop) atomicOr(err, kErrSingular);
  }
  if (stop) return true;
  for (int e = tid; e < n * n; e += CNT) {
    const int i = e / n, j = e - (e / n) * n;
    const T v = (j <= i) ? A[e] : T(0);
    if (Lrow) Lrow[e] = static_cast<double>(v);
    if (Lcol) Lcol[static_cast<int64_t>(j) * n + i] = static_cast<double>(v);
    if (img64) img64[j * np + i] = static_cast<double>(v);
    if (img32) img32[j * np + i] = static_cast<float>(v);
  }
  for (int k = tid; k < n; k += CNT) {
    keep_out[k] = keepv[k];
    invdiag[k] = keepv[k] ? 1.0 / static_cast<double>(A[k * n + k]) : 0.0;
  }
  return true;
}

// FP32 factorisation of the mixed LS step for n <= kTileCholMax, with the trailing matrix
// in registers. Warps 1.. own 4 x 4 tiles of the lower triangle (TPT tiles a thread, tile
// rows and columns 4b..4b+3): at step k they load the 4 + 4 entries of column k they need and
// apply 16 predicated FMAs; an entry of column k+2 is then final but for column k+1's update,
// which warp 0 applies, so it is stored to the column-major buffer Acol. Warp 0 holds column
// k in registers (lane l: rows l + 32q), forms column k+1 from Acol, takes its pivot and
// publishes it to the double-buffered colbuf and to the image img (FP32 or FP64). One
// barrier per column. Every entry receives the same fmaf updates in the same order as in
// the generic FP32 form. Returns false (no factor written) when a pivot is <= tol_scale *
// max diag.
constexpr int kTileCholMax = 160;

template <int TPT, typename TI>
__device__ __forceinline__ bool cholesky_f32_tiles(const double* __restrict__ G, int n,
                                                   double tol_scale, float* Acol,
                                                   double* invdiag, int* keep_out, int* info,
                                                   TI* img, float* gimg32) {
  constexpr int QN = (kTileCholMax + 31) / 32;
  __shared__ float colbuf[2][kTileCholMax];
  __shared__ float s_ldiag[kTileCholMax];
  __shared__ float s_tol;
  __shared__ int s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = n + 1;
  const int nb = (n + 3) >> 2;
  const int ntiles = nb * (nb + 1) / 2;
  // owner tiles and their entries
  float a[TPT][4][4];
  int ti[TPT], tj[TPT];
  if (warp > 0) {
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const int t = (tid - 32) + (CNT - 32) * u;
      int bi = -1, bj = 0;
      if (t < ntiles) {
        bi = static_cast<int>((sqrtf(8.0f * static_cast<float>(t) + 1.0f) - 1.0f) * 0.5f);
        while (bi * (bi + 1) / 2 > t) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        bj = t - bi * (bi + 1) / 2;
      }
      ti[u] = bi * 4;
      tj[u] = bj * 4;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = ti[u] + r, j = tj[u] + c;
          a[u][r][c] = (bi >= 0 && i < n && j <= i)
                           ? static_cast<float>(G[static_cast<int64_t>(j) * n + i]) : 0.0f;
        }
    }
  }
  if (gimg32)
    for (int e = tid; e < n * n; e += CNT) {
      const int i = e / n, j = e - (e / n) * n;
      if (j <= i) {
        const float g = static_cast<float>(G[static_cast<int64_t>(j) * n + i]);
        gimg32[j * np + i] = g;
        gimg32[i * np + j] = g;
      }
    }
  // warp 0: column 0 (final after scaling) and column 1 (raw), max diagonal
  float colv[QN];
  if (warp == 0) {
    float md = 0.0f;
    for (int i = lane; i < n; i += 32)
      md = fmaxf(md, static_cast<float>(G[static_cast<int64_t>(i) * n + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    const float tol = static_cast<float>(tol_scale) * md;
    const float d = static_cast<float>(G[0]);
    const bool ok = d > tol;
    const float inv = ok ? rsqrtf(d) : 0.0f;
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int i = lane + 32 * q;
      float v = 0.0f;
      if (i < n) {
        v = (i == 0) ? d * inv : static_cast<float>(G[i]) * inv;   // G[0][i] = G[i][0]
        colbuf[0][i] = v;
        if (n > 1) Acol[n + i] = (i >= 1) ? static_cast<float>(G[n + i]) : 0.0f;
      }
      colv[q] = v;
    }
    if (lane == 0) {
      s_tol = tol;
      s_stop = ok ? 0 : 1;
      s_ldiag[0] = colv[0];
    }
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int i = lane + 32 * q;
      if (i < n) img[i] = static_cast<TI>(colv[q]);              // column 0 of the image
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (s_stop) break;
    const float* cur = colbuf[k & 1];
    if (warp == 0) {
      if (k + 1 < n) {
        const float lk1 = cur[k + 1];
        float av[QN];
#pragma unroll
        for (int q = 0; q < QN; ++q) {
          const int i = lane + 32 * q;
          av[q] = (i >= k + 1 && i < n) ? fmaf(-colv[q], lk1, Acol[(k + 1) * n + i]) : 0.0f;
        }
        // the pivot row k+1 sits in lane (k+1)%32, slot (k+1)/32
        const int pl = (k + 1) & 31, pq = (k + 1) >> 5;
        float dsel = av[0];
#pragma unroll
        for (int q = 1; q < QN; ++q) dsel = (q == pq) ? av[q] : dsel;
        const float d = __shfl_sync(0xffffffffu, dsel, pl);
        const bool ok = d > s_tol;
        const float inv = ok ? rsqrtf(d) : 0.0f;
        float* nxt = colbuf[(k + 1) & 1];
#pragma unroll
        for (int q = 0; q < QN; ++q) {
          const int i = lane + 32 * q;
          float v = 0.0f;
          if (i >= k + 1 && i < n) {
            v = (i == k + 1) ? d * inv : av[q] * inv;
            nxt[i] = v;
            img[(k + 1) * np + i] = static_cast<TI>(v);
          } else if (i < k + 1) {
            img[(k + 1) * np + i] = TI(0);
          }
          colv[q] = v;
        }
        if (lane == 0) {
          s_ldiag[k + 1] = d * inv;
          if (!ok) s_stop = k + 2;
        }
      }
    } else {
      const int j0 = k + 2;
#pragma unroll
      for (int u = 0; u < TPT; ++u) {
        if (ti[u] + 3 < j0 || tj[u] + 3 < j0) continue;   // tile finished (or none)
        float ci[4], cj[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          ci[r] = (ti[u] + r < n) ? cur[ti[u] + r] : 0.0f;
          cj[r] = (tj[u] + r < n) ? cur[tj[u] + r] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int i = ti[u] + r, j = tj[u] + c;
            if (j >= j0 && j <= i && i < n) {
              a[u][r][c] = fmaf(-ci[r], cj[c], a[u][r][c]);
              if (j == j0) Acol[j * n + i] = a[u][r][c];
            }
          }
      }
    }
    __syncthreads();
  }
  if (s_stop) return false;
  for (int k = tid; k < n; k += CNT) {
    keep_out[k] = 1;
    invdiag[k] = 1.0 / static_cast<double>(s_ldiag[k]);
  }
  if (tid == 0) *info = 0;
  return true;
}

// FP32 first, FP64 if needed: the factorisation of the mixed-precision LS step's normal
// matrix (mode 0, image TI = float). The FP32 attempt accepts the factor only if every pivot
// exceeds tol32 * max diag (so it never drops a column); otherwise the same matrix is factored
// in FP64 with tol64 and the mode's rule. A32 and A64 are the work arrays (they may alias).
// Lrow/Lcol receive the FP64 factor only on the FP64 branch. (The sampling distributions keep
// their FP64 factorisation: FP32 rounding in p would change which indices the inverse CDF
// draws.)
template <typename TI>
__device__ __forceinline__ void cholesky_cta_mixed(const double* __restrict__ G, int n, int mode,
                                                   double tol64, double tol32, float* A32,
                                                   double* A64, double* Lrow, double* Lcol,
                                                   double* invdiag, int* keep_out, int* info,
                                                   unsigned* err, TI* img, float* gimg32) {
  constexpr bool f32img = sizeof(TI) == 4;
  double* img64 = f32img ? nullptr : reinterpret_cast<double*>(img);
  float* img32 = f32img ? reinterpret_cast<float*>(img) : nullptr;
  if (n <= kTileCholMax && img) {
    const int nb = (n + 3) >> 2;
    const bool done = nb * (nb + 1) / 2 <= CNT - 32
        ? cholesky_f32_tiles<1, TI>(G, n, tol32, A32, invdiag, keep_out, info, img, gimg32)
        : cholesky_f32_tiles<2, TI>(G, n, tol32, A32, invdiag, keep_out, info, img, gimg32);
    if (done) return;
  } else if (cholesky_cta<float>(G, n, 0, tol32, A32, nullptr, nullptr, invdiag, keep_out,
                                 info, err, img64, img32, gimg32, false)) {
    return;
  }
  __syncthreads();
  cholesky_cta<double>(G, n, mode, tol64, A64, Lrow, Lcol, invdiag, keep_out, info, err, img64,
                       img32, gimg32, true);
}

}  // namespace trk
