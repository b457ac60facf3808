// p^(n) = ell / sum(ell) and its CDF (eq. for p^(n); the inverse-CDF sampler of Alg. 3
// reads the CDF), and the N(0,1) core initialiser (Sec. 3: cores drawn i.i.d. N(0,1)).
#include "common.cuh"

namespace trk {
namespace {

constexpr int PNT = 1024;

// Exclusive scan of one double per thread over the CTA (fixed order), returns the total.
__device__ __forceinline__ double block_exclusive_scan(double v, double* warp_tot, double* out_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    double t = (lane < PNT / 32) ? warp_tot[lane] : 0.0;
    double ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < PNT / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) *out_total = ti;
  }
  __syncthreads();
  return warp_tot[warp] + inc - v;
}

__global__ void __launch_bounds__(PNT) k_cdf(const double* __restrict__ ell, int64_t I,
                                             double* __restrict__ p, double* __restrict__ cdf,
                                             unsigned* err, const int* __restrict__ skip) {
  if (skip && *skip) return;  // the core was not updated: keep its distribution
  __shared__ double warp_tot[PNT / 32];
  __shared__ double s_total;
  const int t = threadIdx.x;
  const int64_t chunk = (I + PNT - 1) / PNT;
  const int64_t b = t * chunk, e = (b + chunk < I) ? b + chunk : I;
  double s = 0.0;
  for (int64_t i = b; i < e; ++i) s += ell[i];
  block_exclusive_scan(s, warp_tot, &s_total);
  const double total = s_total;
  const bool bad = !(total > 0.0) || !isfinite(total);
  if (bad) {
    for (int64_t i = b; i < e; ++i) {
      p[i] = 1.0 / static_cast<double>(I);
      cdf[i] = static_cast<double>(i + 1) / static_cast<double>(I);
    }
    if (t == 0) atomicOr(err, kErrSingular);
    return;
  }
  double sp = 0.0;
  for (int64_t i = b; i < e; ++i) sp += ell[i] / total;
  __syncthreads();
  double run = block_exclusive_scan(sp, warp_tot, &s_total);
  for (int64_t i = b; i < e; ++i) {
    const double pi = ell[i] / total;
    p[i] = pi;
    run += pi;
    cdf[i] = run;
  }
}

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

cudaError_t launch_cdf(const double* ell, int64_t I, double* p, double* cdf, unsigned* err,
                       cudaStream_t st, const int* skip) {
  k_cdf<<<1, PNT, 0, st>>>(ell, I, p, cdf, err, skip);
  return cudaGetLastError();
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
