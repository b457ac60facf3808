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
constexpr int FSPW = 4;      // samples per warp
constexpr int kStageBytes = 96 * 1024;

// Fused draw + subchain: one warp per sample; lane m draws ring position m (its Philox
// block, inverse CDF in shared-memory copies of p and the CDF), lane 0 forms the weight,
// then the warp multiplies the sampled slices and writes the weighted row of A.
template <typename T>
__global__ void __launch_bounds__(FW * 32) k_sample_chain(SampleArgs sa, ChainArgs ca, int64_t J,
                                                          uint32_t key0, uint32_t key1,
                                                          uint32_t uid_lo, uint32_t uid_hi,
                                                          int32_t* __restrict__ idx,
                                                          double* __restrict__ w,
                                                          T* __restrict__ A, int staged) {
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
  if (!sa.uniform) {
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
  const double wuni = sa.uniform ? uniform_weight(J, sa.I, npos) : 0.0;
  for (int s = 0; s < FSPW; ++s) {
    const int64_t j = (static_cast<int64_t>(blockIdx.x) * FW + warp) * FSPW + s;
    if (j >= J) break;
    int64_t mine = 0;
    double pmine = 1.0;
    if (lane < npos) {
      const double u = draw_uniform(j, lane, key0, key1, uid_lo, uid_hi);
      if (sa.uniform) {
        mine = uniform_index(sa.I[lane], u);
      } else {
        mine = inverse_cdf(cp[lane], pp[lane], sa.I[lane], u);
        pmine = pp[lane][mine];
      }
      idx[j * npos + lane] = static_cast<int32_t>(mine);
    }
    double wj = wuni;
    if (!sa.uniform) {
      double pm[kMaxModes];
      for (int m = 0; m < npos; ++m) pm[m] = __shfl_sync(0xffffffffu, pmine, m);
      wj = sample_weight(J, pm, npos);
    }
    if (lane == 0) w[j] = wj;
    auto index = [&](int m) -> int64_t {
      return static_cast<int64_t>(__shfl_sync(0xffffffffu, static_cast<int>(mine), m));
    };
    warp_slice_chain<T>(ca, index, sS[warp], sG[warp], lane);
    const T scale = static_cast<T>(wj);
    for (int e = lane; e < Lout; e += 32) A[j * Lout + e] = sS[warp][e] * scale;
    __syncwarp();
  }
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
                                void* A, bool f64, cudaStream_t st) {
  if (J <= 0) return cudaSuccess;
  int64_t need = 0;
  if (!sa.uniform)
    for (int m = 0; m < sa.npos; ++m) need += 2 * sa.I[m] * static_cast<int64_t>(sizeof(double));
  const int staged = need <= kStageBytes ? 1 : 0;
  const size_t dyn = staged ? static_cast<size_t>(need) : 0;
  const int64_t per = FW * FSPW;
  const unsigned blocks = static_cast<unsigned>((J + per - 1) / per);
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  const uint32_t u0 = static_cast<uint32_t>(update_id), u1 = static_cast<uint32_t>(update_id >> 32);
  if (f64)
    k_sample_chain<double><<<blocks, FW * 32, dyn, st>>>(sa, ca, J, k0, k1, u0, u1, idx, w,
                                                         static_cast<double*>(A), staged);
  else
    k_sample_chain<float><<<blocks, FW * 32, dyn, st>>>(sa, ca, J, k0, k1, u0, u1, idx, w,
                                                        static_cast<float*>(A), staged);
  return cudaGetLastError();
}

cudaError_t sample_chain_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_sample_chain<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_sample_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kStageBytes);
}

}  // namespace trk
