// Single-problem launch of the triangular solves (trsm_body.cuh): the LS step of Alg. 2
// (row a6) and the leverage rows of Def. 4 (row a1). FP32 instances here, FP64 in
// trsm_f64.cu.
#include "trsm_launch.cuh"

namespace trk {

cudaError_t trsm_run_f32(int n, const double* Lrow, const double* Lcol, const double* invdiag,
                         const int* info, int64_t nvec, const double* rhs, int64_t ld, int mode,
                         const double* M, const float* Limg, const float* Mimg, int Rl, int Rr,
                         double* core_out, double* ell, const CdfEpilogue& ep, cudaStream_t st) {
  return run<float, 1>(n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, Rl, Rr,
                       core_out, ell, ep, st);
}

cudaError_t trsm_f32_attributes() { return attr<float, 1>(); }

cudaError_t launch_trsm(int mode, bool f32, int n, const double* Lrow, const double* Lcol,
                        const double* invdiag, const int* info, int64_t nvec, const double* rhs,
                        int64_t ld, const double* M, int Rl, int Rr, double* core_out,
                        double* ell, cudaStream_t st, const void* Limg, const float* Mimg,
                        const CdfEpilogue* cdf) {
  if (nvec <= 0) return cudaSuccess;
  const CdfEpilogue ep = cdf ? *cdf : CdfEpilogue{};
  if (f32)
    return trsm_run_f32(n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M,
                        static_cast<const float*>(Limg), Mimg, Rl, Rr, core_out, ell, ep, st);
  return trsm_run_f64(n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M,
                      static_cast<const double*>(Limg), Mimg, Rl, Rr, core_out, ell, ep, st);
}

size_t trsm_image_bytes(int n, bool f32) {
  return ((static_cast<size_t>(n) * (n + 1) * (f32 ? 4 : 8) + 15) / 16) * 16;
}

cudaError_t trsm_attributes() {
  cudaError_t e = trsm_f32_attributes();
  if (e != cudaSuccess) return e;
  return trsm_f64_attributes();
}

}  // namespace trk
