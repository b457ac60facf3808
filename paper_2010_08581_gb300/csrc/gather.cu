// Row a4: sampled mode-n fibres of X (Alg. 2, "compute X~ = S X_[n]^T"; Def. 2).
// Y[j][i] = w_j * X(i_0, .., i at mode n, .., i_{N-1}) for the sampled multi-index j.
//
// One warp per sample row; lanes walk the fibre. When the gathered mode is the last
// (contiguous) mode and the row is 16-byte aligned, lanes move 16-byte vectors.
#include "common.cuh"

namespace trk {
namespace {

constexpr int kWarps = 8;

template <typename TX, typename TY>
__global__ void __launch_bounds__(kWarps * 32) k_gather(GatherArgs a,
                                                        const TX* __restrict__ X,
                                                        const int32_t* __restrict__ idx,
                                                        const double* __restrict__ w,
                                                        int64_t J, TY* __restrict__ Y,
                                                        unsigned* err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t In = a.In;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * kWarps + warp; j < J;
       j += static_cast<int64_t>(gridDim.x) * kWarps) {
    int64_t base = 0;
    bool bad = false;
    for (int m = 0; m < a.npos; ++m) {
      const int32_t i = idx[j * a.npos + m];
      bad |= (i < 0) || (static_cast<int64_t>(i) >= a.I[m]);
      base += static_cast<int64_t>(i) * a.stride[m];
    }
    TY* out = Y + j * In;
    if (bad) {
      for (int64_t i = lane; i < In; i += 32) out[i] = TY(0);
      if (lane == 0) atomicOr(err, kErrBadIndex);
      continue;
    }
    const TY s = w ? static_cast<TY>(w[j]) : TY(1);
    const TX* src = X + base;
    constexpr int V = 16 / sizeof(TX);
    if (a.stride_n == 1 && sizeof(TX) == sizeof(TY) &&
        (reinterpret_cast<uintptr_t>(src) % 16 == 0) &&
        (reinterpret_cast<uintptr_t>(out) % 16 == 0)) {
      const int64_t nv = In / V;
      for (int64_t v = lane; v < nv; v += 32) {
        if constexpr (sizeof(TX) == 4) {
          float4 x = __ldg(reinterpret_cast<const float4*>(src) + v);
          float4 y;
          y.x = static_cast<float>(x.x * s); y.y = static_cast<float>(x.y * s);
          y.z = static_cast<float>(x.z * s); y.w = static_cast<float>(x.w * s);
          reinterpret_cast<float4*>(out)[v] = y;
        } else {
          double2 x = __ldg(reinterpret_cast<const double2*>(src) + v);
          double2 y;
          y.x = static_cast<double>(x.x * s); y.y = static_cast<double>(x.y * s);
          reinterpret_cast<double2*>(out)[v] = y;
        }
      }
      for (int64_t i = nv * V + lane; i < In; i += 32)
        out[i] = static_cast<TY>(static_cast<TY>(src[i]) * s);
    } else {
      for (int64_t i = lane; i < In; i += 32)
        out[i] = static_cast<TY>(static_cast<TY>(src[i * a.stride_n]) * s);
    }
  }
}

template <typename TX, typename TY>
cudaError_t run(const GatherArgs& a, const void* X, const int32_t* idx, const double* w,
                int64_t J, void* Y, unsigned* err, cudaStream_t st) {
  int64_t blocks = (J + kWarps - 1) / kWarps;
  if (blocks > sm_count() * 16) blocks = sm_count() * 16;
  k_gather<TX, TY><<<static_cast<unsigned>(blocks), kWarps * 32, 0, st>>>(
      a, static_cast<const TX*>(X), idx, w, J, static_cast<TY*>(Y), err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather(const GatherArgs& a, const void* X, bool x_f64, const int32_t* idx,
                          const double* w, int64_t J, void* Y, bool y_f64, unsigned* err,
                          cudaStream_t st) {
  if (J <= 0) return cudaSuccess;
  if (x_f64 && y_f64) return run<double, double>(a, X, idx, w, J, Y, err, st);
  if (x_f64) return run<double, float>(a, X, idx, w, J, Y, err, st);
  if (y_f64) return run<float, double>(a, X, idx, w, J, Y, err, st);
  return run<float, float>(a, X, idx, w, J, Y, err, st);
}

}  // namespace trk
