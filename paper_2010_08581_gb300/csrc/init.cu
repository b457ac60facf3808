// The N(0,1) core initialiser (Sec. 4: cores drawn i.i.d. N(0,1)).
#include <atomic>

#include "draw.cuh"

namespace trk {
namespace {

// N(0,1) by Philox4x32-10 + Box-Muller, one pair per thread (normal_pair in draw.cuh).
__global__ void k_init_normal(double* __restrict__ out, int64_t count, uint32_t k0, uint32_t k1,
                              uint32_t stream_id, const uint64_t* __restrict__ seed_dev) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (2 * q >= count) return;
  if (seed_dev) {
    const uint64_t s = *seed_dev;
    k0 = static_cast<uint32_t>(s);
    k1 = static_cast<uint32_t>(s >> 32);
  }
  double z0, z1;
  normal_pair(q, stream_id, k0, k1, &z0, &z1);
  out[2 * q] = z0;
  if (2 * q + 1 < count) out[2 * q + 1] = z1;
}

}  // namespace

int sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    dev = -1;
  } else if (const int v = cache[dev].load(std::memory_order_relaxed); v > 0) {
    return v;
  }
  int n = 0;
  if (dev < 0 || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n <= 0) {
    cudaGetLastError();
    return 148;   // a conservative count when no device can be queried
  }
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

cudaError_t launch_init_normal(double* out, int64_t count, uint64_t seed, uint32_t stream_id,
                               const uint64_t* seed_dev, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t pairs = (count + 1) / 2;
  const int threads = 256;
  k_init_normal<<<static_cast<unsigned>((pairs + threads - 1) / threads), threads, 0, st>>>(
      out, count, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), stream_id,
      seed_dev);
  return cudaGetLastError();
}

}  // namespace trk
