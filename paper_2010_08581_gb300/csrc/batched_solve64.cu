// Batched FP64 substitutions: the LS solve of the FP64 path (Alg. 2 LS step) and the
// leverage rows with the fused p / CDF step (Def. 4, eq. for p^(n)).
#include "batched_trsm.cuh"

namespace trk {
namespace {

template <typename T, int NB>
__global__ void __launch_bounds__(TW * 32) kb_solve(const BInst* __restrict__ tab, int step,
                                                    int smem_bytes) {
  extern __shared__ __align__(16) unsigned char sm[];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, 0, false);
  if (!cu.active) return;
  const int n = cu.L;
  const int64_t per = static_cast<int64_t>(TW) * NB;
  const int nctas = static_cast<int>((cu.I + per - 1) / per);
  if (static_cast<int>(blockIdx.y) >= nctas) return;
  const int mode = sizeof(T) == 4 ? 2 : 1;
  const CdfEpilogue none{};
  const bool smem = staged_bytes<T>(n, mode) <= static_cast<size_t>(smem_bytes);
  const bool packed = !smem && packed_bytes<T>(n) <= static_cast<size_t>(smem_bytes);
  trsm_dispatch<T, NB>(smem, packed, sm, blockIdx.y, n, d.Lrow, d.Lcol, d.invdiag, d.info, cu.I,
                       d.BT, n,
                       mode, d.M, static_cast<const T*>(d.limg), d.mimg, cu.Rl, cu.Rr,
                       d.cores[cu.n], nullptr, none, nctas);
}

__global__ void __launch_bounds__(TW * 32) kb_rows(const BInst* __restrict__ tab, int step,
                                                   int init_k, unsigned* err, int smem_bytes,
                                                   int from_core) {
  extern __shared__ __align__(16) unsigned char sm[];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, true);
  if (!cu.active) return;
  const bool tall = cu.I >= cu.L;
  const int n = tall ? cu.L : static_cast<int>(cu.I);
  const double* rhs = tall ? ((cu.init || from_core) ? d.cores[cu.n] : d.BT) : d.L1row;
  const int64_t ld = tall ? cu.L : cu.I;
  const double* Lr = tall ? d.L1row : d.L2row;
  const double* Lc = tall ? d.L1col : d.L2col;
  const double* iv = tall ? d.inv1 : d.inv2;
  const double* im = tall ? d.img1 : d.img2;
  const int nctas = static_cast<int>((cu.I + TW - 1) / TW);
  if (static_cast<int>(blockIdx.y) >= nctas) return;
  const CdfEpilogue ep{d.counter, d.p[cu.n], d.cdf[cu.n], cu.init ? nullptr : d.info, err};
  const bool smem = staged_bytes<double>(n, 0) <= static_cast<size_t>(smem_bytes);
  const bool packed = !smem && packed_bytes<double>(n) <= static_cast<size_t>(smem_bytes);
  trsm_dispatch<double, 1>(smem, packed, sm, blockIdx.y, n, Lr, Lc, iv, nullptr, cu.I, rhs, ld, 0,
                           nullptr,
                           im, nullptr, 1, 1, nullptr, d.ell, ep, nctas);
}

}  // namespace

cudaError_t bl_solve_f64(const BLaunch& b, int step, cudaStream_t st) {
  const int dyn = solve_smem<double>(b.Lmax, 1);
  dim3 grid(b.count, static_cast<unsigned>((b.Imax + TW - 1) / TW));
  kb_solve<double, 1><<<grid, TW * 32, dyn, st>>>(b.tab, step, dyn);
  return cudaGetLastError();
}

cudaError_t bl_leverage_rows(const BLaunch& b, int step, int init_k, unsigned* err,
                             cudaStream_t st) {
  const int nmax = b.n1max > b.n2max ? b.n1max : b.n2max;
  const int dyn = solve_smem<double>(nmax, 0);
  dim3 grid(b.count, static_cast<unsigned>((b.Imax + TW - 1) / TW));
  kb_rows<<<grid, TW * 32, dyn, st>>>(b.tab, step, init_k, err, dyn, b.ls_mode == 1 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t batched_solve64_attributes() {
  cudaError_t e = cudaFuncSetAttribute(kb_solve<double, 1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kb_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
}

}  // namespace trk
