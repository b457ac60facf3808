// Row a2: J i.i.d. draws from q^{!=n} = prod_{j != n} p^(j) (Alg. 3) by inverse CDF, and
// the Def. 5 rescaling w_j = 1 / sqrt(J q(i_j)), or from the uniform distribution (the
// Sec. 5 variant, no distributions read); and the fused draw + sampled-subchain kernel used
// by the driver (rows a2 + a3: Alg. 3 then Alg. 4 for the same samples).
#include "draw.cuh"

namespace trk {
namespace {

// One thread per sample.
__global__ void __launch_bounds__(256) k_sample(SampleArgs a, int64_t J, uint32_t key0,
                                                uint32_t key1, uint32_t uid_lo,
                                                uint32_t uid_hi, int32_t* __restrict__ idx,
                                                double* __restrict__ w) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= J) return;
  if (a.seed_dev) {
    const uint64_t s = *a.seed_dev;
    key0 = static_cast<uint32_t>(s);
    key1 = static_cast<uint32_t>(s >> 32);
  }
  if (a.uniform) {
    for (int m = 0; m < a.npos; ++m) {
      const double u = draw_uniform(j, m, key0, key1, uid_lo, uid_hi);
      idx[j * a.npos + m] = static_cast<int32_t>(uniform_index(a.I[m], u));
    }
    w[j] = uniform_weight(J, a.I, a.npos);
    return;
  }
  double pm[kMaxModes];
  for (int m = 0; m < a.npos; ++m) {
    const double u = draw_uniform(j, m, key0, key1, uid_lo, uid_hi);
    const int64_t i = inverse_cdf(a.cdf[m], a.p[m], a.I[m], u);
    idx[j * a.npos + m] = static_cast<int32_t>(i);
    pm[m] = a.p[m][i];
  }
  w[j] = sample_weight(J, pm, a.npos);
}

constexpr int FW = 8;        // warps per CTA in the fused kernel
constexpr int kStageBytes = 96 * 1024;

// Fibre of sample j at element offset `off` of X (Alg. 2, sketch of X), scaled by w_j:
// the same arithmetic as k_gather (gather.cu), so the fused and stand-alone forms agree bit
// for bit. 16-byte vectors when the gathered mode is contiguous and both rows are aligned.
template <typename T, typename TX>
__device__ __forceinline__ void warp_fibre(const TX* __restrict__ src, int64_t In,
                                           int64_t stride_n, T s, T* __restrict__ out,
                                           int lane) {
  constexpr int V = 16 / sizeof(TX);
  if (stride_n == 1 && sizeof(TX) == sizeof(T) && (reinterpret_cast<uintptr_t>(src) % 16 == 0) &&
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
        const float4 x = __ldg(reinterpret_cast<const float4*>(src) + v);
        float4 y;
        y.x = static_cast<float>(x.x * s); y.y = static_cast<float>(x.y * s);
        y.z = static_cast<float>(x.z * s); y.w = static_cast<float>(x.w * s);
        reinterpret_cast<float4*>(out)[v] = y;
      } else {
        const double2 x = __ldg(reinterpret_cast<const double2*>(src) + v);
        double2 y;
        y.x = static_cast<double>(x.x * s); y.y = static_cast<double>(x.y * s);
        reinterpret_cast<double2*>(out)[v] = y;
      }
    }
    for (int64_t i = nv * V + lane; i < In; i += 32)
      out[i] = static_cast<T>(static_cast<T>(src[i]) * s);
  } else {
    for (int64_t i = lane; i < In; i += 32)
      out[i] = static_cast<T>(static_cast<T>(src[i * stride_n]) * s);
  }
}

// Fused draw + subchain (+ fibre): one warp per sample; lane m draws ring position m (its
// Philox block, inverse CDF in shared-memory copies of p and the CDF), the weight is formed
// from the shuffled probabilities, the warp multiplies the sampled slices and writes the
// weighted row of A and, when Y is given, the weighted fibre of X. One sample per warp keeps
// enough warps resident to cover the latency of the draw, the slice loads and the fibre.
template <typename T, typename TX>
__global__ void __launch_bounds__(FW * 32) k_sample_chain(SampleArgs sa, ChainArgs ca, int64_t J,
                                                          uint32_t key0, uint32_t key1,
                                                          uint32_t uid_lo, uint32_t uid_hi,
                                                          int32_t* __restrict__ idx,
                                                          double* __restrict__ w,
                                                          T* __restrict__ A, int staged,
                                                          GatherArgs ga, const TX* __restrict__ X,
                                                          T* __restrict__ Y) {
  extern __shared__ __align__(16) double fused_smem[];
  __shared__ T sS[FW][kMaxL];
  __shared__ T sG[FW][kMaxL];
  if (sa.seed_dev) {
    const uint64_t s = *sa.seed_dev;
    key0 = static_cast<uint32_t>(s);
    key1 = static_cast<uint32_t>(s >> 32);
  }
  const double* pp[kMaxModes];
  const double* cp[kMaxModes];
  if (!sa.uniform && !sa.given_idx) {   // given (merged) samples read no distribution
    int64_t off = 0;
    for (int m = 0; m < sa.npos; ++m) {
      if (staged) {
        double* dp = fused_smem + off;
        double* dc = dp + sa.I[m];
        for (int64_t e = threadIdx.x; e < sa.I[m]; e += blockDim.x) {
          dp[e] = sa.p[m][e];
          dc[e] = sa.cdf[m][e];
        }
        pp[m] = dp;
        cp[m] = dc;
        off += 2 * sa.I[m];
      } else {
        pp[m] = sa.p[m];
        cp[m] = sa.cdf[m];
      }
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int npos = sa.npos;
  const int Lout = ca.rl[0] * ca.rr[npos - 1];
  const int64_t j = static_cast<int64_t>(blockIdx.x) * FW + warp;
  if (j >= J || (sa.jdev && j >= *sa.jdev)) return;
  int64_t mine = 0;
  double pmine = 1.0;
  int64_t off = 0;
  if (sa.given_idx) {          // merged samples: indices and weights are given
    if (lane < npos) {
      mine = sa.given_idx[j * npos + lane];
      off = mine * ga.stride[lane];
    }
  } else if (lane < npos) {
    const double u = draw_uniform(j, lane, key0, key1, uid_lo, uid_hi);
    if (sa.uniform) {
      mine = uniform_index(sa.I[lane], u);
    } else {
      mine = inverse_cdf(cp[lane], pp[lane], sa.I[lane], u);
      pmine = pp[lane][mine];
    }
    idx[j * npos + lane] = static_cast<int32_t>(mine);
    off = mine * ga.stride[lane];
  }
  double wj;
  if (sa.given_idx) {
    wj = sa.given_w[j];
  } else if (sa.uniform) {
    wj = uniform_weight(J, sa.I, npos);
  } else {
    double pm[kMaxModes];
    for (int m = 0; m < npos; ++m) pm[m] = __shfl_sync(0xffffffffu, pmine, m);
    wj = sample_weight(J, pm, npos);
  }
  if (lane == 0 && !sa.given_idx) w[j] = wj;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
  auto index = [&](int m) -> int64_t {
    return static_cast<int64_t>(__shfl_sync(0xffffffffu, static_cast<int>(mine), m));
  };
  warp_slice_chain<T>(ca, index, sS[warp], sG[warp], lane);
  const T scale = static_cast<T>(wj);
  for (int e = lane; e < Lout; e += 32) A[j * Lout + e] = sS[warp][e] * scale;
  if (Y) warp_fibre<T, TX>(X + off, ga.In, ga.stride_n, scale, Y + j * ga.In, lane);
}

template <typename T, typename TX>
void run_sample_chain(unsigned blocks, size_t dyn, cudaStream_t st, const SampleArgs& sa,
                      const ChainArgs& ca, int64_t J, uint32_t k0, uint32_t k1, uint32_t u0,
                      uint32_t u1, int32_t* idx, double* w, void* A, int staged,
                      const GatherArgs& ga, const void* X, void* Y) {
  k_sample_chain<T, TX><<<blocks, FW * 32, dyn, st>>>(sa, ca, J, k0, k1, u0, u1, idx, w,
                                                      static_cast<T*>(A), staged, ga,
                                                      static_cast<const TX*>(X),
                                                      static_cast<T*>(Y));
}

}  // namespace

cudaError_t launch_sample(const SampleArgs& a, int64_t J, uint64_t seed, uint64_t update_id,
                          int32_t* idx, double* w, cudaStream_t st) {
  if (J <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (J + threads - 1) / threads;
  k_sample<<<static_cast<unsigned>(blocks), threads, 0, st>>>(
      a, J, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32),
      static_cast<uint32_t>(update_id), static_cast<uint32_t>(update_id >> 32), idx, w);
  return cudaGetLastError();
}

cudaError_t launch_sample_chain(const SampleArgs& sa, const ChainArgs& ca, int64_t J,
                                uint64_t seed, uint64_t update_id, int32_t* idx, double* w,
                                void* A, bool f64, cudaStream_t st, const GatherArgs* ga,
                                const void* X, bool x_f64, void* Y) {
  if (J <= 0) return cudaSuccess;
  int64_t need = 0;
  if (!sa.uniform && !sa.given_idx)
    for (int m = 0; m < sa.npos; ++m) need += 2 * sa.I[m] * static_cast<int64_t>(sizeof(double));
  const int staged = (need > 0 && need <= kStageBytes) ? 1 : 0;
  const size_t dyn = staged ? static_cast<size_t>(need) : 0;
  const unsigned blocks = static_cast<unsigned>((J + FW - 1) / FW);
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  const uint32_t u0 = static_cast<uint32_t>(update_id), u1 = static_cast<uint32_t>(update_id >> 32);
  GatherArgs g{};
  if (ga && Y) g = *ga;
  else Y = nullptr;
  if (f64) {
    if (x_f64) run_sample_chain<double, double>(blocks, dyn, st, sa, ca, J, k0, k1, u0, u1, idx,
                                                w, A, staged, g, X, Y);
    else run_sample_chain<double, float>(blocks, dyn, st, sa, ca, J, k0, k1, u0, u1, idx, w, A,
                                         staged, g, X, Y);
  } else {
    if (x_f64) run_sample_chain<float, double>(blocks, dyn, st, sa, ca, J, k0, k1, u0, u1, idx,
                                               w, A, staged, g, X, Y);
    else run_sample_chain<float, float>(blocks, dyn, st, sa, ca, J, k0, k1, u0, u1, idx, w, A,
                                        staged, g, X, Y);
  }
  return cudaGetLastError();
}

cudaError_t sample_chain_attributes() {
  const void* ks[] = {reinterpret_cast<const void*>(k_sample_chain<double, double>),
                      reinterpret_cast<const void*>(k_sample_chain<double, float>),
                      reinterpret_cast<const void*>(k_sample_chain<float, double>),
                      reinterpret_cast<const void*>(k_sample_chain<float, float>)};
  for (const void* k : ks) {
    const cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace trk
