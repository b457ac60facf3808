// Row a2: J i.i.d. draws from q^{!=n} = prod_{j != n} p^(j) (Alg. 3) by inverse CDF, and
// the Def. 3.4 rescaling w_j = 1 / sqrt(J q(i_j)). One thread per sample; the Philox block
// (j, m/2, update_id) serves ring positions m and m+1.
#include "common.cuh"

namespace trk {
namespace {

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
  double q = 1.0;
  u32x4 r{0, 0, 0, 0};
  for (int m = 0; m < a.npos; ++m) {
    if ((m & 1) == 0)
      r = philox4x32_10(u32x4{static_cast<uint32_t>(j), static_cast<uint32_t>(m >> 1), uid_lo,
                              uid_hi},
                        key0, key1);
    const double u = (m & 1) ? u53(r.z, r.w) : u53(r.x, r.y);
    const double* __restrict__ cdf = a.cdf[m];
    const int64_t I = a.I[m];
    // smallest i with u < cdf[i]
    int64_t lo = 0, hi = I;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (u < cdf[mid]) hi = mid; else lo = mid + 1;
    }
    if (lo >= I) {  // rounding left cdf[I-1] <= u: the largest index of positive mass
      lo = I - 1;
      while (lo > 0 && !(a.p[m][lo] > 0.0)) --lo;
    }
    idx[j * a.npos + m] = static_cast<int32_t>(lo);
    q = q * a.p[m][lo];
  }
  w[j] = 1.0 / sqrt(static_cast<double>(J) * q);
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

}  // namespace trk
