// Gram matrices for the Cholesky-based thin QR behind the leverage scores (row a1:
// Def. 4, eq. for p^(n)), and the fixed-order reduction of split partials used by the
// Gram and by the normal-equation contraction (rows a1, a5).
#include "common.cuh"

namespace trk {
namespace {

// ------------------------------------------------------------------------------------
// Gram: partial[s][p][q] = sum_{t in chunk s} X(t, p) X(t, q), tiles with tp <= tq only.
// X(t, p) = A[t*lda + p] (trans = false) or A[p*lda + t] (trans = true).
// ------------------------------------------------------------------------------------
constexpr int GT = 32, GK = 32, GNT = 256;

__global__ void __launch_bounds__(GNT) k_gram(const double* __restrict__ A, int64_t K, int n,
                                              int64_t lda, bool trans, int64_t chunk,
                                              double* __restrict__ partial) {
  __shared__ double P[GK][GT + 1];
  __shared__ double Q[GK][GT + 1];
  const int nt = (n + GT - 1) / GT;
  int tp = 0, rem = blockIdx.x;
  while (rem >= nt - tp) { rem -= nt - tp; ++tp; }
  const int tq = tp + rem;
  const int p0 = tp * GT, q0 = tq * GT;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t k1 = (k0 + chunk < K) ? k0 + chunk : K;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  double acc[4] = {0, 0, 0, 0};
  for (int64_t kb = k0; kb < k1; kb += GK) {
#pragma unroll
    for (int r = 0; r < (GK * GT) / GNT; ++r) {
      const int e = threadIdx.x + r * GNT;
      int kk, col;
      if (!trans) { kk = e / GT; col = e % GT; } else { col = e / GK; kk = e % GK; }
      const int64_t t = kb + kk;
      const int p = p0 + col, q = q0 + col;
      double vp = 0.0, vq = 0.0;
      if (t < k1) {
        if (p < n) vp = trans ? A[p * lda + t] : A[t * lda + p];
        if (q < n) vq = trans ? A[q * lda + t] : A[t * lda + q];
      }
      P[kk][col] = vp;
      Q[kk][col] = vq;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const double b = Q[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += P[kk][ty + 8 * u] * b;
    }
    __syncthreads();
  }
  double* out = partial + static_cast<int64_t>(blockIdx.y) * n * n;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int p = p0 + ty + 8 * u, q = q0 + tx;
    if (p < n && q < n) out[static_cast<int64_t>(p) * n + q] = acc[u];
  }
}

// ------------------------------------------------------------------------------------
// The same Gram (trans = false) from double-float input planes X = hi + lo, in compensated
// FP32 arithmetic on the FP32 pipe (the FP64 pipe runs at about 1/64 of its rate on this GPU):
// each product's leading part and its exact rounding error (FMA) plus the cross terms, then a
// two-sum into a (sum, correction) pair per output. About 47 significant bits, as the
// double-float factorisation that consumes the Gram.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(GNT) k_gram_ff(const float* __restrict__ Ah,
                                                 const float* __restrict__ Al, int64_t K, int n,
                                                 int64_t lda, int64_t chunk,
                                                 double* __restrict__ partial) {
  __shared__ float Ph[GK][GT + 1], Pl[GK][GT + 1];
  __shared__ float Qh[GK][GT + 1], Ql[GK][GT + 1];
  const int nt = (n + GT - 1) / GT;
  int tp = 0, rem = blockIdx.x;
  while (rem >= nt - tp) { rem -= nt - tp; ++tp; }
  const int tq = tp + rem;
  const int p0 = tp * GT, q0 = tq * GT;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t k1 = (k0 + chunk < K) ? k0 + chunk : K;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  float sum[4] = {0.f, 0.f, 0.f, 0.f}, cor[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t kb = k0; kb < k1; kb += GK) {
#pragma unroll
    for (int r = 0; r < (GK * GT) / GNT; ++r) {
      const int e = threadIdx.x + r * GNT;
      const int kk = e / GT, col = e % GT;
      const int64_t t = kb + kk;
      const int p = p0 + col, q = q0 + col;
      const bool okp = t < k1 && p < n, okq = t < k1 && q < n;
      Ph[kk][col] = okp ? Ah[t * lda + p] : 0.f;
      Pl[kk][col] = okp ? Al[t * lda + p] : 0.f;
      Qh[kk][col] = okq ? Ah[t * lda + q] : 0.f;
      Ql[kk][col] = okq ? Al[t * lda + q] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const float yh = Qh[kk][tx], yl = Ql[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float xh = Ph[kk][ty + 8 * u], xl = Pl[kk][ty + 8 * u];
        const float pr = xh * yh;
        float er = fmaf(xh, yh, -pr);
        er = fmaf(xh, yl, er);
        er = fmaf(xl, yh, er);
        const float t2 = sum[u] + pr;
        const float bv = t2 - sum[u];
        const float ts = (sum[u] - (t2 - bv)) + (pr - bv);
        sum[u] = t2;
        cor[u] += ts + er;
      }
    }
    __syncthreads();
  }
  double* out = partial + static_cast<int64_t>(blockIdx.y) * n * n;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int p = p0 + ty + 8 * u, q = q0 + tx;
    if (p < n && q < n)
      out[static_cast<int64_t>(p) * n + q] = static_cast<double>(sum[u]) + static_cast<double>(cor[u]);
  }
}

// ------------------------------------------------------------------------------------
// Fixed-order reduction of split partials (s = 0, 1, ..., splits-1) into FP64 (FP64
// partials: FP64 sum; FP32 partials: compensated FP32 sum, then FP64).
// Columns c < c_split go to out1[r*ld1 + c]; columns c >= c_split go transposed to
// out2[(c - c_split)*ld2 + r]. One element per thread, loads coalesced along c.
// ------------------------------------------------------------------------------------
template <typename TP>
__global__ void __launch_bounds__(256) k_reduce(const TP* __restrict__ partial, int splits,
                                                int64_t pstride, int64_t pld, int64_t nrows,
                                                int64_t ncols, int64_t c_split,
                                                double* __restrict__ out1, int64_t ld1,
                                                double* __restrict__ out2, int64_t ld2,
                                                ReduceSplit sp) {
  const int64_t total = nrows * ncols;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / ncols, c = e - (e / ncols) * ncols;
    const TP* src = partial + r * pld + c;
    double s;
    if constexpr (sizeof(TP) == 4) {
      // FP32 partials: Neumaier-compensated FP32 sum in the fixed order (the FP64 pipe is
      // about 1/64 of the FP32 rate on this GPU), one conversion at the end.
      float hi = 0.f, lo = 0.f;
      int q = 0;
      for (; q + 8 <= splits; q += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = src[(q + u) * pstride];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float t = hi + v[u];
          lo += (fabsf(hi) >= fabsf(v[u])) ? (hi - t) + v[u] : (v[u] - t) + hi;
          hi = t;
        }
      }
      for (; q < splits; ++q) {
        const float v = src[q * pstride];
        const float t = hi + v;
        lo += (fabsf(hi) >= fabsf(v)) ? (hi - t) + v : (v - t) + hi;
        hi = t;
      }
      s = static_cast<double>(hi) + static_cast<double>(lo);
      if (c < c_split) {   // the FP32 value of out1 is the rounded pair sum
        const float f = hi + lo;
        if (sp.hi && c >= r) sp.hi[r * sp.lda + c] = f;
        if (sp.img) sp.img[r * sp.np + c] = f;
      }
    } else {
      s = 0.0;
      int q = 0;
      for (; q + 8 <= splits; q += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = static_cast<double>(src[(q + u) * pstride]);
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
      }
      for (; q < splits; ++q) s += static_cast<double>(src[q * pstride]);
      if (c < c_split && c >= r && sp.hi) {   // double-float split: hi + lo = s
        const float h = static_cast<float>(s);
        sp.hi[r * sp.lda + c] = h;
        if (sp.lo) sp.lo[r * sp.lda + c] = static_cast<float>(s - static_cast<double>(h));
      }
    }
    if (c < c_split) {
      out1[r * ld1 + c] = s;
    } else {
      const int64_t o = (c - c_split) * ld2 + r;
      out2[o] = s;
      if (sp.t_hi) {   // double-float planes of the transposed block (the Gram's input)
        const float h = static_cast<float>(s);
        sp.t_hi[o] = h;
        sp.t_lo[o] = static_cast<float>(s - static_cast<double>(h));
      }
    }
  }
}

int plan_splits(int64_t K, int tiles, int min_chunk, int64_t* chunk) {
  int64_t s = (2 * sm_count() + tiles - 1) / tiles;
  const int64_t maxs = (K + min_chunk - 1) / min_chunk;
  if (s > maxs) s = maxs;
  if (s < 1) s = 1;
  int64_t c = (K + s - 1) / s;
  c = (c + GK - 1) / GK * GK;
  s = (K + c - 1) / c;
  if (s < 1) s = 1;
  *chunk = c;
  return static_cast<int>(s);
}

}  // namespace

size_t gram_workspace(int64_t rows, int cols, bool trans, int* splits) {
  const int64_t K = trans ? cols : rows;
  const int n = trans ? static_cast<int>(rows) : cols;
  const int nt = (n + GT - 1) / GT;
  int64_t chunk;
  *splits = plan_splits(K, nt * (nt + 1) / 2, GK, &chunk);
  return static_cast<size_t>(*splits) * n * n * sizeof(double);
}

cudaError_t launch_gram(const double* A, int64_t rows, int cols, int64_t lda, bool trans,
                        double* partial, int splits, cudaStream_t st) {
  const int64_t K = trans ? cols : rows;
  const int n = trans ? static_cast<int>(rows) : cols;
  const int nt = (n + GT - 1) / GT;
  int64_t chunk;
  const int s = plan_splits(K, nt * (nt + 1) / 2, GK, &chunk);
  if (s != splits) return cudaErrorInvalidValue;
  dim3 grid(nt * (nt + 1) / 2, s);
  k_gram<<<grid, GNT, 0, st>>>(A, K, n, lda, trans, chunk, partial);
  return cudaGetLastError();
}

cudaError_t launch_gram_ff(const float* Ah, const float* Al, int64_t rows, int cols,
                           int64_t lda, double* partial, int splits, cudaStream_t st) {
  const int n = cols;
  const int nt = (n + GT - 1) / GT;
  int64_t chunk;
  const int s = plan_splits(rows, nt * (nt + 1) / 2, GK, &chunk);
  if (s != splits) return cudaErrorInvalidValue;
  dim3 grid(nt * (nt + 1) / 2, s);
  k_gram_ff<<<grid, GNT, 0, st>>>(Ah, Al, rows, n, lda, chunk, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const void* partial, bool partial_f32, int splits, int64_t pstride,
                          int64_t pld, int64_t nrows, int64_t ncols, int64_t c_split,
                          double* out1, int64_t ld1, double* out2, int64_t ld2,
                          cudaStream_t st, const ReduceSplit& split) {
  const int64_t total = nrows * ncols;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > sm_count() * 16) blocks = sm_count() * 16;
  if (partial_f32)
    k_reduce<float><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        static_cast<const float*>(partial), splits, pstride, pld, nrows, ncols, c_split, out1,
        ld1, out2, ld2, split);
  else
    k_reduce<double><<<static_cast<unsigned>(blocks), 256, 0, st>>>(
        static_cast<const double*>(partial), splits, pstride, pld, nrows, ncols, c_split, out1,
        ld1, out2, ld2, split);
  return cudaGetLastError();
}

}  // namespace trk
