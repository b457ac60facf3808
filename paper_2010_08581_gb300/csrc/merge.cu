// Merging repeated draws (Sec. 4.2): the J sampled multi-indices of one update are reduced
// to one row per distinct multi-index, in the order of first occurrence, with weight
// sqrt(count) * w (Def. 5's rescaling depends only on the multi-index, so the c copies of a
// row contribute c * w^2 a a^T to the normal equations, as the merged row does).
//
// One CTA: the ring linear index of every sample (first listed mode fastest) is sorted with
// its sample number by a bitonic sort in shared memory; the first element of every run of
// equal keys carries the smallest sample number, i.e. the first occurrence, and the run's
// length. A fixed-order block scan over the first-occurrence flags, in sample order, gives
// each distinct multi-index its output position.
#include "common.cuh"

namespace trk {
namespace {

constexpr int MT = 1024;

__global__ void __launch_bounds__(MT) k_merge(const int32_t* __restrict__ idx,
                                              const double* __restrict__ w, int J, int npos,
                                              MergeArgs a, int32_t* __restrict__ idx_out,
                                              double* __restrict__ w_out,
                                              int64_t* __restrict__ J_out) {
  extern __shared__ __align__(16) unsigned char msm[];
  const int Jp = a.Jpow2;
  uint64_t* key = reinterpret_cast<uint64_t*>(msm);
  int* sj = reinterpret_cast<int*>(key + Jp);
  int* cnt = sj + Jp;                 // [J]: run length at the first occurrence, else 0
  __shared__ int s_part[MT];
  __shared__ int s_total;
  const int t = threadIdx.x;
  for (int e = t; e < Jp; e += MT) {
    uint64_t k = ~0ull;
    if (e < J) {
      k = 0;
      for (int m = 0; m < npos; ++m)
        k += static_cast<uint64_t>(idx[static_cast<int64_t>(e) * npos + m]) * a.stride[m];
    }
    key[e] = k;
    sj[e] = e;
  }
  for (int e = t; e < J; e += MT) cnt[e] = 0;
  __syncthreads();
  // bitonic sort of (key, sample) pairs, ascending
  for (int size = 2; size <= Jp; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int e = t; e < Jp / 2; e += MT) {
        const int lo = 2 * e - (e & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t kl = key[lo], kh = key[hi];
        const int jl = sj[lo], jh = sj[hi];
        const bool gt = kl > kh || (kl == kh && jl > jh);
        if (gt == up) {
          key[lo] = kh; key[hi] = kl;
          sj[lo] = jh; sj[hi] = jl;
        }
      }
      __syncthreads();
    }
  }
  // run heads: the first occurrence of each distinct key and its count
  for (int e = t; e < J; e += MT) {
    if (e == 0 || key[e] != key[e - 1]) {
      int r = e + 1;
      while (r < J && key[r] == key[e]) ++r;
      cnt[sj[e]] = r - e;
    }
  }
  __syncthreads();
  // output positions: exclusive scan of (cnt > 0) in sample order, contiguous chunks
  const int chunk = (J + MT - 1) / MT;
  const int b = t * chunk, e1 = b + chunk < J ? b + chunk : J;
  int c = 0;
  for (int e = b; e < e1; ++e) c += cnt[e] > 0 ? 1 : 0;
  s_part[t] = c;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int q = 0; q < MT; ++q) { const int v = s_part[q]; s_part[q] = run; run += v; }
    s_total = run;
  }
  __syncthreads();
  int pos = s_part[t];
  for (int e = b; e < e1; ++e) {
    const int n = cnt[e];
    if (n > 0) {
      for (int m = 0; m < npos; ++m)
        idx_out[static_cast<int64_t>(pos) * npos + m] = idx[static_cast<int64_t>(e) * npos + m];
      w_out[pos] = w[e] * sqrt(static_cast<double>(n));
      ++pos;
    }
  }
  if (t == 0) *J_out = s_total;
}

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

size_t merge_smem(int J) {
  const int Jp = pow2_at_least(J);
  return static_cast<size_t>(Jp) * (8 + 4) + static_cast<size_t>(J) * 4;
}

}  // namespace

bool merge_fits(int64_t J, int npos, const int64_t* I, MergeArgs* a) {
  if (J < 1 || J > kMergeMaxJ) return false;
  uint64_t s = 1;
  for (int m = 0; m < npos; ++m) {
    if (I[m] < 1) return false;
    a->stride[m] = s;
    const uint64_t next = s * static_cast<uint64_t>(I[m]);
    if (next / static_cast<uint64_t>(I[m]) != s || next >= (1ull << 63)) return false;
    s = next;
  }
  a->Jpow2 = pow2_at_least(static_cast<int>(J));
  return true;
}

cudaError_t launch_merge(const int32_t* idx, const double* w, int64_t J, int npos,
                         const MergeArgs& a, int32_t* idx_out, double* w_out, int64_t* J_out,
                         cudaStream_t st) {
  if (J < 1 || J > kMergeMaxJ) return cudaErrorInvalidValue;
  k_merge<<<1, MT, merge_smem(static_cast<int>(J)), st>>>(idx, w, static_cast<int>(J), npos, a,
                                                         idx_out, w_out, J_out);
  return cudaGetLastError();
}

cudaError_t merge_attributes() {
  return cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(merge_smem(kMergeMaxJ)));
}

}  // namespace trk
