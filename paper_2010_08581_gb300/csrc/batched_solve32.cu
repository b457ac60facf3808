// Batched LS solve of the mixed-precision path (FP32 substitutions with one refinement
// step, Alg. 2 LS step), writing each instance's new core.
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

}  // namespace

cudaError_t bl_solve_f32(const BLaunch& b, int step, cudaStream_t st) {
  const int dyn = solve_smem<float>(b.Lmax, 2);
  dim3 grid(b.count, static_cast<unsigned>((b.Imax + 2 * TW - 1) / (2 * TW)));
  kb_solve<float, 2><<<grid, TW * 32, dyn, st>>>(b.tab, step, dyn);
  return cudaGetLastError();
}

cudaError_t batched_solve32_attributes() {
  return cudaFuncSetAttribute(kb_solve<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kDyn);
}

}  // namespace trk
