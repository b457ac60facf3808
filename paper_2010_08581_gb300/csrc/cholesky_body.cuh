// One-CTA FP64 Cholesky factorisation G = L L^T (n <= 256), shared by the single-problem
// kernel and the batched kernel. Used for the normal matrix of the sampled LS (row a6,
// Alg. 2 LS step) and for the R factor of the Cholesky-based thin QR behind the leverage
// scores (row a1).
//
// Right-looking with one column of look-ahead. At step k column k is final; warp 0 applies
// column k's update to column k+1 only, takes its pivot (FP64 rsqrt) and scales it, while
// warps 1.. apply column k's rank-1 update to the trailing triangle of columns >= k+2
// (its (m+1)m/2 entries spread evenly over the threads). One barrier per column. A is the
// n x n work array (shared memory, or the Lrow output itself).
//
// Every update is one fused multiply-add, a_ij = fma(-l_ik, l_jk, a_ij), so that the cluster
// kernel (cholesky_cluster.cu), which applies the same updates in the same order, gives the
// same factor.
//
// mode 0 (solve): a pivot <= tol_scale * max diag stops the factorisation (*info = column
// + 1, singular bit). mode 1 (leverage): such a column is dropped (zero, keep = 0).
// Besides L (row- and column-major) the kernel can write padded images that the
// triangular-solve kernels copy straight into shared memory: img[c*(n+1) + r] = L[r][c] in
// FP64 and/or FP32, and the FP32 image of the symmetric input matrix.
#pragma once

#include "common.cuh"

namespace trk {

constexpr int CNT = 512;

__device__ __forceinline__ void cholesky_cta(const double* __restrict__ G, int n, int mode,
                                             double tol_scale, double* A, double* Lrow,
                                             double* Lcol, double* invdiag, int* keep_out,
                                             int* info, unsigned* err, double* img64,
                                             float* img32, float* gimg32) {
  __shared__ double colbuf[2][kMaxL];
  __shared__ int keepv[kMaxL];
  __shared__ double s_tol;
  __shared__ int s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = n + 1;
  for (int e = tid; e < n * n; e += CNT) {
    const int i = e / n, j = e - (e / n) * n;
    if (j <= i) {
      const double g = G[static_cast<int64_t>(j) * n + i];
      A[e] = g;
      if (gimg32) {
        gimg32[j * np + i] = static_cast<float>(g);
        gimg32[i * np + j] = static_cast<float>(g);
      }
    } else {
      A[e] = 0.0;
    }
  }
  __syncthreads();
  if (warp == 0) {
    double md = 0.0;
    for (int i = lane; i < n; i += 32) md = fmax(md, A[i * n + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
    const double tol = tol_scale * md;
    const double d = A[0];
    const bool ok = d > tol;                  // false for NaN and non-positive pivots
    const double inv = ok ? rsqrt(d) : 0.0;
    for (int i = lane; i < n; i += 32) {
      const double v = ok ? ((i == 0) ? d * inv : A[i * n] * inv) : 0.0;
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
    const double* cur = colbuf[k & 1];
    double* nxt = colbuf[(k + 1) & 1];
    const bool kp = keepv[k] != 0;
    if (warp == 0) {
      if (k + 1 < n) {
        // column k+1: a_i = A[i][k+1] - L[i][k] L[k+1][k]; pivot; scale
        const double lk1 = cur[k + 1];
        double a[kMaxL / 32];
#pragma unroll
        for (int q = 0; q < kMaxL / 32; ++q) {
          const int i = k + 1 + lane + 32 * q;
          a[q] = 0.0;
          if (i < n) a[q] = kp ? fma(-cur[i], lk1, A[i * n + k + 1]) : A[i * n + k + 1];
        }
        const double d = __shfl_sync(0xffffffffu, a[0], 0);   // row k+1: lane 0, q = 0
        const bool ok = d > s_tol;
        const double inv = ok ? rsqrt(d) : 0.0;
#pragma unroll
        for (int q = 0; q < kMaxL / 32; ++q) {
          const int i = k + 1 + lane + 32 * q;
          if (i < n) {
            const double v = ok ? ((i == k + 1) ? d * inv : a[q] * inv) : 0.0;
            A[i * n + k + 1] = v;
            nxt[i] = v;
          }
        }
        if (lane == 0) {
          keepv[k + 1] = ok ? 1 : 0;
          if (!ok && mode == 0) s_stop = k + 2;
        }
      }
    } else if (kp) {
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
    if (img64) img64[j * np + i] = v;
    if (img32) img32[j * np + i] = static_cast<float>(v);
  }
  for (int k = tid; k < n; k += CNT) {
    keep_out[k] = keepv[k];
    invdiag[k] = keepv[k] ? 1.0 / A[k * n + k] : 0.0;
  }
}


}  // namespace trk
