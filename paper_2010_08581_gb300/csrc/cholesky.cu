// FP64 Cholesky factorisation G = L L^T of an n x n symmetric matrix (n <= 256) in one CTA.
// Used for the normal matrix of the sampled LS (row a6, Alg. 2 LS step) and for the R
// factor of the Cholesky-based thin QR behind the leverage scores (row a1).
//
// Right-looking, one column per step: scale column k by 1/sqrt(pivot), then update the
// trailing lower triangle, whose (m+1)m/2 entries are spread evenly over all threads.
// The thread that updates the next diagonal entry also decides the next pivot, so each
// column costs two barriers. The matrix lives in shared memory when n*n*8 <= 200 KB,
// otherwise in place in the Lrow output.
#include "common.cuh"

namespace trk {
namespace {

constexpr int CNT = 512;

__device__ __forceinline__ void decide_pivot(double d, double tol, int k, int mode, double* s_inv,
                                             int* s_keep, int* keepv, int* s_stop) {
  const bool ok = d > tol;  // false for NaN and for non-positive pivots
  s_keep[k & 1] = ok ? 1 : 0;
  s_inv[k & 1] = ok ? 1.0 / sqrt(d) : 0.0;
  keepv[k] = ok ? 1 : 0;
  if (!ok && mode == 0) *s_stop = k + 1;
}

__global__ void __launch_bounds__(CNT) k_cholesky(const double* __restrict__ G, int n, int mode,
                                                  double tol_scale, double* Lrow, double* Lcol,
                                                  double* invdiag, int* keep_out, int* info,
                                                  unsigned* err, int use_smem) {
  extern __shared__ double smem[];
  __shared__ double colk[kMaxL];
  __shared__ int keepv[kMaxL];
  __shared__ double s_inv[2];
  __shared__ int s_keep[2];
  __shared__ double s_tol;
  __shared__ int s_stop;
  double* A = use_smem ? smem : Lrow;
  const int tid = threadIdx.x;
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
    decide_pivot(A[0], s_tol, 0, mode, s_inv, s_keep, keepv, &s_stop);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (s_stop) break;
    const bool kp = s_keep[k & 1] != 0;
    const double inv = s_inv[k & 1];
    // column k: L_kk = d * (1/sqrt d) = sqrt d, L_ik = A_ik / sqrt d
    for (int i = k + tid; i < n; i += CNT) {
      const double v = kp ? A[i * n + k] * inv : 0.0;
      A[i * n + k] = v;
      colk[i] = v;
    }
    __syncthreads();
    const int m = n - k - 1;
    if (kp) {
      const int P = m * (m + 1) / 2;
      for (int e = tid; e < P; e += CNT) {
        int ii = static_cast<int>((sqrtf(8.0f * static_cast<float>(e) + 1.0f) - 1.0f) * 0.5f);
        while (ii * (ii + 1) / 2 > e) --ii;
        while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
        const int jj = e - ii * (ii + 1) / 2;
        const int i = k + 1 + ii, j = k + 1 + jj;
        const double nv = A[i * n + j] - colk[i] * colk[j];
        A[i * n + j] = nv;
        if (e == 0) decide_pivot(nv, s_tol, k + 1, mode, s_inv, s_keep, keepv, &s_stop);
      }
    } else if (tid == 0 && m > 0) {
      decide_pivot(A[(k + 1) * n + k + 1], s_tol, k + 1, mode, s_inv, s_keep, keepv, &s_stop);
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
  }
  for (int k = tid; k < n; k += CNT) {
    keep_out[k] = keepv[k];
    invdiag[k] = keepv[k] ? 1.0 / A[k * n + k] : 0.0;
  }
}

}  // namespace

cudaError_t launch_cholesky(const double* G, int n, int mode, double tol_scale, double* Lrow,
                            double* Lcol, double* invdiag, int* keep, int* info, unsigned* err,
                            cudaStream_t st) {
  const size_t bytes = static_cast<size_t>(n) * n * sizeof(double);
  const int use_smem = bytes <= 200 * 1024 ? 1 : 0;
  const size_t dyn = use_smem ? bytes : 0;
  k_cholesky<<<1, CNT, dyn, st>>>(G, n, mode, tol_scale, Lrow, Lcol, invdiag, keep, info, err,
                                  use_smem);
  return cudaGetLastError();
}

cudaError_t cholesky_attributes() {
  return cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace trk
