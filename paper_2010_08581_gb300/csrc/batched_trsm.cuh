// Launch-time choice of the triangular-solve variant for the batched solve kernels
// (batched_solve32.cu, batched_solve64.cu).
#pragma once

#include "batched_kern.cuh"
#include "trsm_body.cuh"

namespace trk {
namespace {

// ------------------------------------------------------------------------------------
// Triangular solves: the LS solve (mode 2 mixed / mode 1 FP64) writing the new core, and
// the leverage rows with the fused p / CDF step.
// ------------------------------------------------------------------------------------
// Runtime choice of the register rows (QN = ceil(n/32)) and of shared-memory staging:
// n <= 128 always fits padded; beyond that the packed layout when it fits (`packed`), else
// the image stays in global memory.
template <typename T, int NB>
__device__ __forceinline__ void trsm_dispatch(bool smem, bool packed, unsigned char* sm,
                                              int64_t cta, int n,
                                              const double* Lrow, const double* Lcol,
                                              const double* invdiag, const int* info,
                                              int64_t nvec, const double* rhs, int64_t ld,
                                              int mode, const double* M, const T* Limg,
                                              const float* Mimg, int Rl, int Rr,
                                              double* core_out, double* ell,
                                              const CdfEpilogue& ep, int nctas) {
#define TB_ARGS sm, cta, n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Limg, Mimg, Rl, Rr, \
                core_out, ell, ep, nctas
  switch ((n + 31) / 32) {
    case 1: trsm_cta<T, 1, NB, true>(TB_ARGS); break;
    case 2: trsm_cta<T, 2, NB, true>(TB_ARGS); break;
    case 3: trsm_cta<T, 3, NB, true>(TB_ARGS); break;
    case 4: trsm_cta<T, 4, NB, true>(TB_ARGS); break;
    case 5:
      if (smem) trsm_cta<T, 5, NB, true>(TB_ARGS);
      else if (packed) trsm_cta<T, 5, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 5, NB, false>(TB_ARGS);
      break;
    case 6:
      if (packed) trsm_cta<T, 6, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 6, NB, false>(TB_ARGS);
      break;
    case 7:
      if (packed) trsm_cta<T, 7, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 7, NB, false>(TB_ARGS);
      break;
    case 8:
      if (packed) trsm_cta<T, 8, NB, true, true>(TB_ARGS);
      else trsm_cta<T, 8, NB, false>(TB_ARGS);
      break;
    default: break;
  }
#undef TB_ARGS
}

// Dynamic shared memory for the solve kernels: enough for every instance that takes the
// shared-memory path (every n <= 128 does; n >= 161 never does).
template <typename T>
int solve_smem(int nmax, int mode) {
  const int n = nmax < 160 ? nmax : 160;
  size_t need = staged_bytes<T>(n, mode);
  const size_t pk = packed_bytes<T>(nmax);
  if (nmax > 128 && pk <= static_cast<size_t>(kDyn) && pk > need) need = pk;
  return need <= static_cast<size_t>(kDyn) ? static_cast<int>(need) : kDyn;
}

}  // namespace
}  // namespace trk
