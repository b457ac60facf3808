// Row a3: sampled subchain rows (Alg. 4; Def. 3). For sample j the lateral slices
// G^(n+1)(:, i_{n+1}, :) ... G^(n-1)(:, i_{n-1}, :) are multiplied in ring order into an
// Rr_n x Rl_n matrix S_j (paper's R_n x R_{n-1}); row j of the sketch is w_j * S_j flattened
// row-major, i.e. column a + Rl_n * b holds S_j[b][a] (the paper's overline{r_{n-1} r_n}).
//
// One warp per sample: the running product lives in shared memory (<= 16 x 16), each lane
// owns up to 8 entries of the next product, and every slice is read once, contiguously.
#include "draw.cuh"

namespace trk {
namespace {

constexpr int kWarps = 8;
constexpr int kMaxEnt = 256;  // ranks <= 16

template <typename T>
__global__ void __launch_bounds__(kWarps * 32) k_subchain(ChainArgs a,
                                                          const int32_t* __restrict__ idx,
                                                          const double* __restrict__ w,
                                                          int64_t J, T* __restrict__ A,
                                                          unsigned* err) {
  __shared__ T sS[kWarps][kMaxEnt];
  __shared__ T sG[kWarps][kMaxEnt];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = static_cast<int64_t>(blockIdx.x) * kWarps + warp;
  if (j >= J) return;
  T* S = sS[warp];
  T* G = sG[warp];
  const int Lout = a.rl[0] * a.rr[a.npos - 1];

  // Validate this sample's indices.
  bool bad = false;
  for (int m = 0; m < a.npos; ++m) {
    const int32_t i = idx[j * a.npos + m];
    bad |= (i < 0) || (static_cast<int64_t>(i) >= a.I[m]);
  }
  if (bad) {
    for (int e = lane; e < Lout; e += 32) A[j * Lout + e] = T(0);
    if (lane == 0) atomicOr(err, kErrBadIndex);
    return;
  }

  auto index = [&](int m) -> int64_t { return idx[j * a.npos + m]; };
  warp_slice_chain<T>(a, index, S, G, lane);
  __syncwarp();
  const T scale = w ? static_cast<T>(w[j]) : T(1);
  for (int e = lane; e < Lout; e += 32) A[j * Lout + e] = S[e] * scale;
}

}  // namespace

cudaError_t launch_subchain(const ChainArgs& a, const int32_t* idx, const double* w,
                            int64_t J, void* A, bool f64, unsigned* err, cudaStream_t st) {
  if (J <= 0) return cudaSuccess;
  const int64_t blocks = (J + kWarps - 1) / kWarps;
  if (f64)
    k_subchain<double><<<static_cast<unsigned>(blocks), kWarps * 32, 0, st>>>(
        a, idx, w, J, static_cast<double*>(A), err);
  else
    k_subchain<float><<<static_cast<unsigned>(blocks), kWarps * 32, 0, st>>>(
        a, idx, w, J, static_cast<float*>(A), err);
  return cudaGetLastError();
}

}  // namespace trk
