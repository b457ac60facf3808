// FP64 instances of the single-problem triangular solves (trsm_launch.cuh): the FP64 LS
// step of Alg. 2 and the leverage rows of Def. 4.
#include "trsm_launch.cuh"

namespace trk {

cudaError_t trsm_run_f64(int n, const double* Lrow, const double* Lcol, const double* invdiag,
                         const int* info, int64_t nvec, const double* rhs, int64_t ld, int mode,
                         const double* M, const double* Limg, const float* Mimg, int Rl, int Rr,
                         double* core_out, double* ell, const CdfEpilogue& ep, cudaStream_t st) {
  return run<double, 1>(n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, Rl, Rr,
                        core_out, ell, ep, st);
}

cudaError_t trsm_f64_attributes() { return attr<double, 1>(); }

}  // namespace trk
