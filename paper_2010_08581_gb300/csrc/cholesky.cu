// Single-problem launch of the one-CTA FP64 Cholesky factorisation (cholesky_body.cuh).
#include <cstdlib>

#include "cholesky_body.cuh"

namespace trk {
namespace {

__global__ void __launch_bounds__(CNT) k_cholesky(const double* __restrict__ G, int n, int mode,
                                                  double tol_scale, double* Lrow, double* Lcol,
                                                  double* invdiag, int* keep_out, int* info,
                                                  unsigned* err, int use_smem,
                                                  double* img64, float* img32, float* gimg32) {
  extern __shared__ double smem[];
  cholesky_cta(G, n, mode, tol_scale, use_smem ? smem : Lrow, Lrow, Lcol, invdiag, keep_out,
               info, err, img64, img32, gimg32);
}

}  // namespace

bool cholesky_cluster_fits(int n);
cudaError_t launch_cholesky_cluster(const double* G, int n, int mode, double tol_scale,
                                    double* Lrow, double* Lcol, double* invdiag, int* keep,
                                    int* info, unsigned* err, cudaStream_t st, double* img64,
                                    float* img32, float* gimg32);

// The cluster form for n <= 144 unless TRALS_CHOL_ONE_CTA=1 selects the one-CTA kernel
// (both give the same factors; the switch exists for comparisons).
bool use_cluster_cholesky(int n) {
  static const bool one_cta = [] {
    const char* e = getenv("TRALS_CHOL_ONE_CTA");
    return e && e[0] == '1';
  }();
  return !one_cta && cholesky_cluster_fits(n);
}

cudaError_t launch_cholesky(const double* G, int n, int mode, double tol_scale, double* Lrow,
                            double* Lcol, double* invdiag, int* keep, int* info, unsigned* err,
                            cudaStream_t st, double* img64, float* img32, float* gimg32) {
  if (use_cluster_cholesky(n))
    return launch_cholesky_cluster(G, n, mode, tol_scale, Lrow, Lcol, invdiag, keep, info, err,
                                   st, img64, img32, gimg32);
  const size_t bytes = static_cast<size_t>(n) * n * sizeof(double);
  const int use_smem = bytes <= 200 * 1024 ? 1 : 0;
  const size_t dyn = use_smem ? bytes : 0;
  k_cholesky<<<1, CNT, dyn, st>>>(G, n, mode, tol_scale, Lrow, Lcol, invdiag, keep, info, err,
                                  use_smem, img64, img32, gimg32);
  return cudaGetLastError();
}

cudaError_t cholesky_cluster_attributes();

cudaError_t cholesky_attributes() {
  const cudaError_t e =
      cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cholesky_cluster_attributes();
}

}  // namespace trk
