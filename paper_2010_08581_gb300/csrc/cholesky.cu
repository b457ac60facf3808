// FP64 Cholesky factorisation G = L L^T of an n x n symmetric matrix (n <= 256) in one CTA.
// Used for the normal matrix of the sampled LS (row a6, Alg. 2 LS step) and for the R
// factor of the Cholesky-based thin QR behind the leverage scores (row a1).
//
// Right-looking with one column of look-ahead. At step k column k is final; warp 0 applies
// column k's update to column k+1 only, takes its pivot (FP64 rsqrt) and scales it, while
// warps 1.. apply column k's rank-1 update to the trailing triangle of columns >= k+2
// (its (m+1)m/2 entries spread evenly over the threads). One barrier per column. The
// matrix lives in shared memory when n*n*8 <= 200 KB, otherwise in place in Lrow.
//
// Besides L (row- and column-major) the kernel can write padded images that the
// triangular-solve kernel copies straight into shared memory: img[c*(n+1) + r] = L[r][c]
// in FP64 and/or FP32, and the FP32 image of the symmetric input matrix.
#include "common.cuh"

namespace trk {
namespace {

constexpr int CNT = 512;

__global__ void __launch_bounds__(CNT) k_cholesky(const double* __restrict__ G, int n, int mode,
                                                  double tol_scale, double* Lrow, double* Lcol,
                                                  double* invdiag, int* keep_out, int* info,
                                                  unsigned* err, int use_smem,
                                                  double* img64, float* img32, float* gimg32) {
  extern __shared__ double smem[];
  __shared__ double colbuf[2][kMaxL];
  __shared__ int keepv[kMaxL];
  __shared__ double s_tol;
  __shared__ int s_stop;
  double* A = use_smem ? smem : Lrow;
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
          if (i < n) a[q] = kp ? A[i * n + k + 1] - cur[i] * lk1 : A[i * n + k + 1];
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
        A[i * n + j] -= cur[i] * cur[j];
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

}  // namespace

cudaError_t launch_cholesky(const double* G, int n, int mode, double tol_scale, double* Lrow,
                            double* Lcol, double* invdiag, int* keep, int* info, unsigned* err,
                            cudaStream_t st, double* img64, float* img32, float* gimg32) {
  const size_t bytes = static_cast<size_t>(n) * n * sizeof(double);
  const int use_smem = bytes <= 200 * 1024 ? 1 : 0;
  const size_t dyn = use_smem ? bytes : 0;
  k_cholesky<<<1, CNT, dyn, st>>>(G, n, mode, tol_scale, Lrow, Lcol, invdiag, keep, info, err,
                                  use_smem, img64, img32, gimg32);
  return cudaGetLastError();
}

cudaError_t cholesky_attributes() {
  return cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace trk
