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
      int64_t v = lane;
      if constexpr (sizeof(TX) == 4) {
        // four 16-byte loads in flight per lane before their stores
        for (; v + 96 < nv; v += 128) {
          float4 x[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = __ldg(reinterpret_cast<const float4*>(src) + v + 32 * u);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float4 y;
            y.x = static_cast<float>(x[u].x * s); y.y = static_cast<float>(x[u].y * s);
            y.z = static_cast<float>(x[u].z * s); y.w = static_cast<float>(x[u].w * s);
            reinterpret_cast<float4*>(out)[v + 32 * u] = y;
          }
        }
      }
      for (; v < nv; v += 32) {
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

// X viewed as [P_pre][I_n][P_post] (row-major) copied to [P_pre][P_post][I_n]: mode n moved
// last, so that its fibres are contiguous. 32 x 32 tiles through shared memory (padded against
// bank conflicts): reads coalesced along P_post, writes along I_n.
constexpr int TT = 32, TR = 8;

template <typename TX>
__global__ void __launch_bounds__(TT * TR) k_mode_last(const TX* __restrict__ X, int64_t In,
                                                       int64_t Post, int64_t tiles_n,
                                                       int64_t tiles_p, TX* __restrict__ out) {
  __shared__ TX tile[TT][TT + 1];
  const int64_t b = blockIdx.x;
  const int64_t per = tiles_n * tiles_p;
  const int64_t pre = b / per;
  const int64_t r = b - pre * per;
  const int64_t tn = r / tiles_p, tp = r - tn * tiles_p;
  const int64_t i0 = tn * TT, q0 = tp * TT;
  const TX* src = X + pre * In * Post;
  TX* dst = out + pre * In * Post;
  const int tx = threadIdx.x & (TT - 1), ty = threadIdx.x / TT;
#pragma unroll
  for (int k = 0; k < TT; k += TR) {
    const int64_t i = i0 + ty + k, q = q0 + tx;
    if (i < In && q < Post) tile[ty + k][tx] = src[i * Post + q];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < TT; k += TR) {
    const int64_t q = q0 + ty + k, i = i0 + tx;
    if (i < In && q < Post) dst[q * In + i] = tile[tx][ty + k];
  }
}

// FP32 with 16-byte accesses: 64 x 64 tiles, 256 threads; float4 loads along P_post and
// float4 stores along I_n when both extents are multiples of 4 (else the kernel above).
constexpr int T4 = 64;

__global__ void __launch_bounds__(256) k_mode_last4(const float* __restrict__ X, int64_t In,
                                                    int64_t Post, int64_t tiles_n,
                                                    int64_t tiles_p, float* __restrict__ out) {
  __shared__ float tile[T4][T4 + 1];
  const int64_t b = blockIdx.x;
  const int64_t per = tiles_n * tiles_p;
  const int64_t pre = b / per;
  const int64_t r = b - pre * per;
  const int64_t tn = r / tiles_p, tp = r - tn * tiles_p;
  const int64_t i0 = tn * T4, q0 = tp * T4;
  const float* src = X + pre * In * Post;
  float* dst = out + pre * In * Post;
  const int t = threadIdx.x, c4 = 4 * (t & 15), r0 = t >> 4;
#pragma unroll
  for (int k = 0; k < T4; k += 16) {
    const int64_t i = i0 + r0 + k, q = q0 + c4;
    if (i < In && q < Post) {   // Post % 4 == 0: the whole vector is in range
      const float4 v = __ldg(reinterpret_cast<const float4*>(src + i * Post + q));
      tile[r0 + k][c4] = v.x; tile[r0 + k][c4 + 1] = v.y;
      tile[r0 + k][c4 + 2] = v.z; tile[r0 + k][c4 + 3] = v.w;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < T4; k += 16) {
    const int64_t q = q0 + r0 + k, i = i0 + c4;
    if (i < In && q < Post) {   // In % 4 == 0
      const int qq = r0 + k;
      *reinterpret_cast<float4*>(dst + q * In + i) =
          make_float4(tile[c4][qq], tile[c4 + 1][qq], tile[c4 + 2][qq], tile[c4 + 3][qq]);
    }
  }
}

}  // namespace

cudaError_t launch_mode_last(const void* X, bool x_f64, int64_t pre, int64_t In, int64_t post,
                             void* out, cudaStream_t st) {
  if (pre <= 0 || In <= 0 || post <= 0) return cudaSuccess;
  if (!x_f64 && In % 4 == 0 && post % 4 == 0 &&
      reinterpret_cast<uintptr_t>(X) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 16 == 0) {
    const int64_t tn4 = (In + T4 - 1) / T4, tp4 = (post + T4 - 1) / T4;
    const int64_t b4 = pre * tn4 * tp4;
    if (b4 > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_mode_last4<<<static_cast<unsigned>(b4), 256, 0, st>>>(static_cast<const float*>(X), In,
                                                            post, tn4, tp4,
                                                            static_cast<float*>(out));
    return cudaGetLastError();
  }
  const int64_t tn = (In + TT - 1) / TT, tp = (post + TT - 1) / TT;
  const int64_t blocks = pre * tn * tp;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (x_f64)
    k_mode_last<double><<<static_cast<unsigned>(blocks), TT * TR, 0, st>>>(
        static_cast<const double*>(X), In, post, tn, tp, static_cast<double*>(out));
  else
    k_mode_last<float><<<static_cast<unsigned>(blocks), TT * TR, 0, st>>>(
        static_cast<const float*>(X), In, post, tn, tp, static_cast<float*>(out));
  return cudaGetLastError();
}

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
