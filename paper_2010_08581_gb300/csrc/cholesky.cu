// Single-problem launches of the one-CTA Cholesky factorisation (cholesky_body.cuh) for
// the leverage scores of Def. 4 (row a1) and the LS step of Alg. 2 (row a6): FP64, the
// mixed LS step's FP32-then-FP64 form, and the double-float leverage form.
#include "chol_inv.cuh"
#include "cholesky_body.cuh"

namespace trk {
namespace {

constexpr int kCholDyn = 200 * 1024;   // the work matrix, when it fits

__global__ void __launch_bounds__(CNT) k_cholesky(const double* __restrict__ G, int n, int mode,
                                                  double tol_scale, double* Lrow, double* Lcol,
                                                  double* invdiag, int* keep_out, int* info,
                                                  unsigned* err, int use_smem,
                                                  double* img64, float* img32, float* gimg32) {
  extern __shared__ double smem[];
  cholesky_cta(G, n, mode, tol_scale, use_smem ? smem : Lrow, Lrow, Lcol, invdiag, keep_out,
               info, err, img64, img32, gimg32);
}

// The mixed-precision LS step: FP32 factorisation, FP64 when an FP32 pivot is too small.
template <typename TI>
__global__ void __launch_bounds__(CNT) k_cholesky_mixed(const double* __restrict__ G, int n,
                                                        int mode, double tol64, double tol32,
                                                        double* Lrow, double* Lcol,
                                                        double* invdiag, int* keep_out,
                                                        int* info, unsigned* err, int dyn_bytes,
                                                        TI* img, float* gimg32,
                                                        const float* pre,
                                                        const int* __restrict__ skip_if) {
  extern __shared__ double smem[];
  if (skip_if && *skip_if) return;   // the factor and its inverse are formed already
  // A contraction whose bounded wait expired left no valid normal equations: report
  // info = -1 so that the solve leaves the core unchanged (the error bit is already set).
  if (err && (*reinterpret_cast<volatile unsigned*>(err) & kErrTimeout)) {
    if (threadIdx.x == 0) *info = -1;
    return;
  }
  const int64_t nn = static_cast<int64_t>(n) * n;
  float* A32 = nn * 4 <= dyn_bytes ? reinterpret_cast<float*>(smem) : reinterpret_cast<float*>(Lrow);
  double* A64 = nn * 8 <= dyn_bytes ? smem : Lrow;
  cholesky_cta_mixed<TI>(G, n, mode, tol64, tol32, A32, A64, Lrow, Lcol, invdiag, keep_out, info,
                         err, img, gimg32, A32 == reinterpret_cast<float*>(smem) ? pre : nullptr);
}

// The mixed-precision LS step's FP32 factor and its inverse in one CTA (chol_inv_tiles) from
// the reduction's FP32 work array pre; on success wimg, keep, *info = 0 and *fast = 1,
// otherwise *fast = 0 and nothing else (k_cholesky_mixed then runs). A contraction whose
// bounded wait expired gives *info = -1 and *fast = 1 (nothing to factor).
__global__ void __launch_bounds__(kCiMaxThreads) k_chol_inv_solve(int n, float tol_scale,
                                                                  const float* __restrict__ pre,
                                                                  int lda, float* __restrict__ wimg,
                                                                  int* __restrict__ keep,
                                                                  int* __restrict__ info,
                                                                  const unsigned* err,
                                                                  int* __restrict__ fast) {
  __shared__ CiShared cs;
  if (err && (*reinterpret_cast<const volatile unsigned*>(err) & kErrTimeout)) {
    if (threadIdx.x == 0) {
      *info = -1;
      *fast = 1;
    }
    return;
  }
  const bool ok = chol_inv_tiles(n, tol_scale, pre, lda, wimg, cs);
  if (ok)
    for (int k = threadIdx.x; k < n; k += blockDim.x) keep[k] = 1;
  if (threadIdx.x == 0) {
    if (ok) *info = 0;
    *fast = ok ? 1 : 0;
  }
}

// The mixed-precision drivers' leverage Gram (tall, mode 1): double-float, FP64 if needed.
__global__ void __launch_bounds__(CNT) k_cholesky_lev_mixed(const double* __restrict__ G, int n,
                                                            double tol64, double tolff,
                                                            double* Lrow, double* Lcol,
                                                            double* invdiag, int* keep_out,
                                                            int* info, unsigned* err,
                                                            int dyn_bytes, double* img64,
                                                            const float* pre_hi,
                                                            const float* pre_lo,
                                                            const int* run_if) {
  extern __shared__ double smem[];
  if (run_if && *run_if == 0) return;
  const int64_t nn = static_cast<int64_t>(n) * n;
  float* Aff = panel_floats<FFOps>(n) * 4 <= dyn_bytes ? reinterpret_cast<float*>(smem) : nullptr;
  double* A64 = nn * 8 <= dyn_bytes ? smem : Lrow;
  cholesky_cta_lev_mixed<4>(G, n, tol64, tolff, Aff, A64, Lrow, Lcol, invdiag, keep_out, info,
                            err, img64, pre_hi, pre_lo);
}

// img64 = hi + lo from the two FP32 planes when the factorisation left them (*info == 2).
__global__ void __launch_bounds__(256) k_ff_image(const float* __restrict__ hi,
                                                  const float* __restrict__ lo, int64_t count,
                                                  const int* __restrict__ info,
                                                  double* __restrict__ img64,
                                                  const int* __restrict__ run_if) {
  if ((run_if && *run_if == 0) || *info != 2) return;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    img64[e] = static_cast<double>(hi[e]) + static_cast<double>(lo[e]);
}

}  // namespace

cudaError_t launch_ff_image(const double* Lrow, const double* Lcol, int n, const int* info,
                            double* img64, cudaStream_t st, const int* run_if) {
  const int64_t count = static_cast<int64_t>(n) * (n + 1);
  const unsigned blocks = static_cast<unsigned>((count + 255) / 256 < sm_count() ? (count + 255) / 256 : sm_count());
  k_ff_image<<<blocks, 256, 0, st>>>(reinterpret_cast<const float*>(Lrow),
                                     reinterpret_cast<const float*>(Lcol), count, info, img64,
                                     run_if);
  return cudaGetLastError();
}

cudaError_t launch_cholesky_lev_mixed(const double* G, int n, double tol64, double tolff,
                                      double* Lrow, double* Lcol, double* invdiag, int* keep,
                                      int* info, unsigned* err, cudaStream_t st, double* img64,
                                      const float* pre_hi, const float* pre_lo,
                                      const int* run_if) {
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t ff = static_cast<size_t>(panel_floats<FFOps>(n)) * 4;
  const size_t want = nn * 8 > ff ? nn * 8 : ff;
  const size_t dyn = want <= kCholDyn ? want : (nn * 8 <= kCholDyn ? nn * 8 : 0);
  k_cholesky_lev_mixed<<<1, CNT, dyn, st>>>(G, n, tol64, tolff, Lrow, Lcol, invdiag, keep, info,
                                            err, static_cast<int>(dyn), img64, pre_hi, pre_lo,
                                            run_if);
  return cudaGetLastError();
}

cudaError_t launch_cholesky_mixed(const double* G, int n, int mode, double tol64, double tol32,
                                  double* Lrow, double* Lcol, double* invdiag, int* keep,
                                  int* info, unsigned* err, cudaStream_t st, float* img32,
                                  float* gimg32, const float* pre, float* wimg, int* fast) {
  const size_t nn = static_cast<size_t>(n) * n;
  const size_t dyn = nn * 8 <= kCholDyn ? nn * 8 : (nn * 4 <= kCholDyn ? nn * 4 : 0);
  const bool tiles = wimg && fast && pre && n >= 4 && n <= kCiMaxN;
  if (tiles) {
    k_chol_inv_solve<<<1, chol_inv_threads(n), 0, st>>>(n, static_cast<float>(tol32), pre,
                                                        (n + 3) & ~3, wimg, keep, info, err, fast);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_cholesky_mixed<float><<<1, CNT, dyn, st>>>(G, n, mode, tol64, tol32, Lrow, Lcol, invdiag, keep,
                                               info, err, static_cast<int>(dyn), img32, gimg32,
                                               pre, tiles ? fast : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_cholesky(const double* G, int n, int mode, double tol_scale, double* Lrow,
                            double* Lcol, double* invdiag, int* keep, int* info, unsigned* err,
                            cudaStream_t st, double* img64, float* img32, float* gimg32) {
  const size_t bytes = static_cast<size_t>(n) * n * sizeof(double);
  const int use_smem = bytes <= kCholDyn ? 1 : 0;
  const size_t dyn = use_smem ? bytes : 0;
  k_cholesky<<<1, CNT, dyn, st>>>(G, n, mode, tol_scale, Lrow, Lcol, invdiag, keep, info, err,
                                  use_smem, img64, img32, gimg32);
  return cudaGetLastError();
}

cudaError_t cholesky_attributes() {
  cudaError_t e =
      cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholDyn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_cholesky_mixed<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kCholDyn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_cholesky_lev_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kCholDyn);
}

}  // namespace trk
