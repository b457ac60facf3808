// The N(0,1) core initialiser (Sec. 3: cores drawn i.i.d. N(0,1)).
#include "common.cuh"

namespace trk {
namespace {

// ------------------------------------------------------------------------------------
// N(0,1) by Philox4x32-10 + Box-Muller (Box & Muller, 1958): pair q uses counter
// (q lo, q hi, stream_id, 0x4E4F524D), two 53-bit uniforms u1, u2; r = sqrt(-2 ln(1-u1)),
// (r cos 2 pi u2, r sin 2 pi u2).
// ------------------------------------------------------------------------------------
__global__ void k_init_normal(double* __restrict__ out, int64_t count, uint32_t k0, uint32_t k1,
                              uint32_t stream_id, const uint64_t* __restrict__ seed_dev) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (2 * q >= count) return;
  if (seed_dev) {
    const uint64_t s = *seed_dev;
    k0 = static_cast<uint32_t>(s);
    k1 = static_cast<uint32_t>(s >> 32);
  }
  const u32x4 r = philox4x32_10(u32x4{static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                      stream_id, 0x4E4F524Du},
                                k0, k1);
  const double u1 = u53(r.x, r.y), u2 = u53(r.z, r.w);
  const double rad = sqrt(-2.0 * log1p(-u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  out[2 * q] = rad * c;
  if (2 * q + 1 < count) out[2 * q + 1] = rad * s;
}

}  // namespace

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
