// Device helpers shared by the sampler kernels (row a2: Alg. 3 and Def. 5) and the
// slice-chain kernels (row a3: Alg. 4), so that the per-stage entry points and the fused
// driver kernel compute bit-identical results.
#pragma once

#include "common.cuh"

namespace trk {

// Uniform of sample j at ring position m: Philox4x32-10 block (j, m/2, update_id), words
// (2(m%2), 2(m%2)+1) as (hi, lo), top 53 bits.
__device__ __forceinline__ double draw_uniform(int64_t j, int m, uint32_t k0, uint32_t k1,
                                               uint32_t uid_lo, uint32_t uid_hi) {
  const u32x4 r = philox4x32_10(
      u32x4{static_cast<uint32_t>(j), static_cast<uint32_t>(m >> 1), uid_lo, uid_hi}, k0, k1);
  return (m & 1) ? u53(r.z, r.w) : u53(r.x, r.y);
}

// N(0,1) pair q of the core initialiser: Philox4x32-10 counter (q lo, q hi, stream_id,
// 0x4E4F524D), two 53-bit uniforms u1, u2; r = sqrt(-2 ln(1-u1)); (r cos 2 pi u2,
// r sin 2 pi u2) (Box & Muller, 1958).
__device__ __forceinline__ void normal_pair(int64_t q, uint32_t stream_id, uint32_t k0,
                                            uint32_t k1, double* z0, double* z1) {
  const u32x4 r = philox4x32_10(u32x4{static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32),
                                      stream_id, 0x4E4F524Du},
                                k0, k1);
  const double u1 = u53(r.x, r.y), u2 = u53(r.z, r.w);
  const double rad = sqrt(-2.0 * log1p(-u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  *z0 = rad * c;
  *z1 = rad * s;
}

// Smallest i with u < cdf[i]; if rounding leaves cdf[I-1] <= u, the largest i with p > 0.
__device__ __forceinline__ int64_t inverse_cdf(const double* cdf, const double* p, int64_t I,
                                               double u) {
  int64_t lo = 0, hi = I;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (u < cdf[mid]) hi = mid; else lo = mid + 1;
  }
  if (lo >= I) {
    lo = I - 1;
    while (lo > 0 && !(p[lo] > 0.0)) --lo;
  }
  return lo;
}

// Uniform sampling (the Sec. 5 alternative to leverage scores): index floor(u * I) of a
// uniform draw on {0, ..., I-1}, clamped to I-1 should the product round up to I.
__device__ __forceinline__ int64_t uniform_index(int64_t I, double u) {
  const double x = floor(__dmul_rn(u, static_cast<double>(I)));
  const int64_t i = static_cast<int64_t>(x);
  return i < I ? i : I - 1;
}

// Weight of every uniform sample, 1 / sqrt(J q) with q = 1 / P: sqrt(P / J), P the product
// of the sampled modes' sizes taken in ring order.
__device__ __forceinline__ double uniform_weight(int64_t J, const int64_t* I, int npos) {
  double P = 1.0;
  for (int m = 0; m < npos; ++m) P = __dmul_rn(P, static_cast<double>(I[m]));
  return sqrt(P / static_cast<double>(J));
}

// w = 1 / sqrt(J * prod_m p_m) with the product taken in ring order m = 0, 1, ...
__device__ __forceinline__ double sample_weight(int64_t J, const double* pm, int npos) {
  double q = 1.0;
  for (int m = 0; m < npos; ++m) q = q * pm[m];
  return 1.0 / sqrt(static_cast<double>(J) * q);
}

// One warp multiplies the sampled lateral slices in ring order into S (row-major,
// R0 x cols, <= 256 entries) held in shared memory; G is a second 256-entry buffer.
// index(m) returns the sampled index at ring position m. Returns the final column count.
template <typename T, typename IndexFn>
__device__ __forceinline__ int warp_slice_chain(const ChainArgs& a, IndexFn index, T* S, T* G,
                                                int lane) {
  {
    const int64_t i = index(0);
    const int ent = a.rl[0] * a.rr[0];
    const double* src = a.core[0] + i * ent;
    for (int e = lane; e < ent; e += 32) S[e] = static_cast<T>(src[e]);
  }
  const int R0 = a.rl[0];
  int cols = a.rr[0];
  for (int m = 1; m < a.npos; ++m) {
    const int64_t i = index(m);
    const int rr = a.rr[m];
    const int ent = cols * rr;
    const double* src = a.core[m] + i * ent;
    for (int e = lane; e < ent; e += 32) G[e] = static_cast<T>(src[e]);
    __syncwarp();
    T acc[kMaxL / 32];
    const int outs = R0 * rr;
#pragma unroll
    for (int q = 0; q < kMaxL / 32; ++q) {
      const int e = lane + 32 * q;
      T s = T(0);
      if (e < outs) {
        const int r = e / rr, c = e - r * rr;
        for (int t = 0; t < cols; ++t) s += S[r * cols + t] * G[t * rr + c];
      }
      acc[q] = s;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kMaxL / 32; ++q) {
      const int e = lane + 32 * q;
      if (e < outs) S[e] = acc[q];
    }
    __syncwarp();
    cols = rr;
  }
  __syncwarp();
  return cols;
}

}  // namespace trk
