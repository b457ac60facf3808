// Single-problem launch templates of the triangular solves (trsm_body.cuh), instantiated
// per arithmetic type in trsm.cu (FP32) and trsm_f64.cu (FP64).
#pragma once

#include "trsm_body.cuh"

namespace trk {
namespace {

template <typename T, int QN, int NB, bool SMEM, bool PACK = false>
__global__ void __launch_bounds__(TW * 32) k_trsm(int n, const double* __restrict__ Lrow,
                                                  const double* __restrict__ Lcol,
                                                  const double* __restrict__ invdiag,
                                                  const int* __restrict__ info, int64_t nvec,
                                                  const double* __restrict__ rhs, int64_t ld,
                                                  int mode, const double* __restrict__ M,
                                                  const T* __restrict__ Limg,
                                                  const float* __restrict__ Mimg, int Rl, int Rr,
                                                  double* __restrict__ core_out,
                                                  double* __restrict__ ell, CdfEpilogue ep) {
  extern __shared__ __align__(16) unsigned char trsm_smem[];
  trsm_cta<T, QN, NB, SMEM, PACK>(trsm_smem, blockIdx.x, n, Lrow, Lcol, invdiag, info, nvec, rhs, ld,
                            mode, M, Limg, Mimg, Rl, Rr, core_out, ell, ep, gridDim.x);
}

template <typename T, int QN, int NB>
cudaError_t run_q(int n, const double* Lrow, const double* Lcol, const double* invdiag,
                  const int* info, int64_t nvec, const double* rhs, int64_t ld, int mode,
                  const double* M, const T* Limg, const float* Mimg, int Rl, int Rr,
                  double* core_out, double* ell, const CdfEpilogue& ep, cudaStream_t st) {
  const size_t staged = staged_bytes<T>(n, mode);
  const int64_t per_cta = static_cast<int64_t>(TW) * NB;
  const unsigned blocks = static_cast<unsigned>((nvec + per_cta - 1) / per_cta);
  // n <= 128 (QN <= 4) always fits in shared memory padded and n >= 161 (QN >= 6) never
  // does; beyond the padded image the packed lower triangle when it fits.
  if constexpr (QN <= 5) {
    if (staged <= 200 * 1024) {
      k_trsm<T, QN, NB, true><<<blocks, TW * 32, staged, st>>>(
          n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, Rl, Rr, core_out,
          ell, ep);
      return cudaGetLastError();
    }
  }
  if constexpr (QN >= 5) {
    const size_t pb = packed_bytes<T>(n);
    if (pb <= 200 * 1024) {
      k_trsm<T, QN, NB, true, true><<<blocks, TW * 32, pb, st>>>(
          n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, Rl, Rr, core_out, ell,
          ep);
      return cudaGetLastError();
    }
    k_trsm<T, QN, NB, false><<<blocks, TW * 32, kMaxL * sizeof(T), st>>>(
        n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, Rl, Rr, core_out, ell,
        ep);
  }
  return cudaGetLastError();
}

template <typename T, int NB>
cudaError_t run(int n, const double* Lrow, const double* Lcol, const double* invdiag,
                const int* info, int64_t nvec, const double* rhs, int64_t ld, int mode,
                const double* M, const T* Limg, const float* Mimg, int Rl, int Rr,
                double* core_out, double* ell, const CdfEpilogue& ep, cudaStream_t st) {
  switch ((n + 31) / 32) {
#define TRSM_CASE(q)                                                                        \
  case q:                                                                                   \
    return run_q<T, q, NB>(n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, \
                           Rl, Rr, core_out, ell, ep, st);
    TRSM_CASE(1) TRSM_CASE(2) TRSM_CASE(3) TRSM_CASE(4)
    TRSM_CASE(5) TRSM_CASE(6) TRSM_CASE(7) TRSM_CASE(8)
#undef TRSM_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int QN, int NB>
cudaError_t attr_q() {
  cudaError_t e = cudaSuccess;
  if constexpr (QN <= 5)
    e = cudaFuncSetAttribute(k_trsm<T, QN, NB, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  if constexpr (QN >= 5) {
    e = cudaFuncSetAttribute(k_trsm<T, QN, NB, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_trsm<T, QN, NB, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  return e;
}

template <typename T, int NB>
cudaError_t attr() {
  cudaError_t e;
  if ((e = attr_q<T, 1, NB>()) != cudaSuccess) return e;
  if ((e = attr_q<T, 2, NB>()) != cudaSuccess) return e;
  if ((e = attr_q<T, 3, NB>()) != cudaSuccess) return e;
  if ((e = attr_q<T, 4, NB>()) != cudaSuccess) return e;
  if ((e = attr_q<T, 5, NB>()) != cudaSuccess) return e;
  if ((e = attr_q<T, 6, NB>()) != cudaSuccess) return e;
  if ((e = attr_q<T, 7, NB>()) != cudaSuccess) return e;
  return attr_q<T, 8, NB>();
}

}  // namespace

// The FP32 and FP64 halves of launch_trsm and of its attribute set-up.
cudaError_t trsm_run_f32(int n, const double* Lrow, const double* Lcol, const double* invdiag,
                         const int* info, int64_t nvec, const double* rhs, int64_t ld, int mode,
                         const double* M, const float* Limg, const float* Mimg, int Rl, int Rr,
                         double* core_out, double* ell, const CdfEpilogue& ep, cudaStream_t st);
cudaError_t trsm_run_f64(int n, const double* Lrow, const double* Lcol, const double* invdiag,
                         const int* info, int64_t nvec, const double* rhs, int64_t ld, int mode,
                         const double* M, const double* Limg, const float* Mimg, int Rl, int Rr,
                         double* core_out, double* ell, const CdfEpilogue& ep, cudaStream_t st);
cudaError_t trsm_f32_attributes();
cudaError_t trsm_f64_attributes();

}  // namespace trk
