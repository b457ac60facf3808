// FP32 Cholesky factor L of a symmetric positive definite n x n matrix K (n <= 128) and its
// inverse W = L^-1, formed together by one CTA with one barrier per block of 4 columns
// (blocked right-looking elimination; the inverse by the block recurrence
// W_II = L_II^-1, W_IJ = -L_II^-1 sum_{J <= M < I} L_IM W_MJ).
//
// Thread t owns the 4 x 4 tile (bi, bj), bi >= bj, t = bi (bi + 1) / 2 + bj, of the working
// matrix in registers: the tile holds A (the trailing matrix) until step K = bj, then R (the
// partial sum of the inverse's recurrence), and W_{bi,bj} from step bi on. Step K:
//   W_KK = L_KK^-1 of the diagonal block, formed at the end of step K - 1 by the owner of
//   tile (K, K) and read from shared memory by every thread; with L_IK = P_I W_KK^T (P_I the
//   column block K of A, rows of block I) and Y = W_KK S,
//     bj > K:  A_{bi,bj} -= L_{bi,K} L_{bj,K}^T     (S = P_bj^T)
//     bj = K:  R_{bi,K}   = -L_{bi,K} W_KK          (S = I)
//     bj < K:  R_{bi,bj} -= L_{bi,K} W_{K,bj}       (S = R_{K,bj}, W_{K,bj} = W_KK R_{K,bj})
//   for bi > K, one code path for the three cases; the tiles of block row K become
//   W_{K,bj} = W_KK R_{K,bj} (W_KK itself on the diagonal).
// At the end of step K the owners of tile column K + 1 publish their A tiles (the next
// column block), the owners of tile row K + 1 their R tiles (transposed), and the owner of
// tile (K + 1, K + 1) factors its block and publishes W_{K+1,K+1}; all double-buffered.
// Only the lower triangle of K is read: K[i][j] = pre[j * lda + i], i >= j.
#pragma once
#include "common.cuh"

namespace trk {

constexpr int kCiMaxN = 128;
constexpr int kCiMaxThreads = 544;   // 528 tiles at n = 128, in whole warps

__host__ __device__ inline int chol_inv_threads(int n) {
  const int nb = (n + 3) >> 2;
  return (nb * (nb + 1) / 2 + 31) / 32 * 32;
}

struct CiShared {
  float4 P[2][kCiMaxN / 4][4];   // column block K of A: [tile row][row r] = (c = 0..3)
  float4 R[2][kCiMaxN / 4][4];   // row block K of R, transposed: [tile column][column c]
  float4 W[2][4];                // W_KK by rows (zeros above the diagonal)
  float4 Id[4];
  int ok[2];
  float tol;
};

namespace ci {

__device__ __forceinline__ void ld(const float4* s, float (&m)[4][4]) {
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const float4 v = s[x];
    m[x][0] = v.x; m[x][1] = v.y; m[x][2] = v.z; m[x][3] = v.w;
  }
}
__device__ __forceinline__ void st(float4* s, const float (&m)[4][4]) {
#pragma unroll
  for (int x = 0; x < 4; ++x) s[x] = make_float4(m[x][0], m[x][1], m[x][2], m[x][3]);
}
__device__ __forceinline__ void st_t(float4* s, const float (&m)[4][4]) {
#pragma unroll
  for (int y = 0; y < 4; ++y) s[y] = make_float4(m[0][y], m[1][y], m[2][y], m[3][y]);
}

// Cholesky of the 4 x 4 block d (lower triangle; rows m with 4K + m >= n are padding and get
// a unit pivot) and W = L^-1 with zeros above the diagonal. False when a real pivot is <= tol.
__device__ __forceinline__ bool factor_block(const float (&d)[4][4], int K, int n, float tol,
                                             float (&w)[4][4]) {
  float l[4][4], rr[4];
  bool ok = true;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float p = d[m][m];
#pragma unroll
    for (int q = 0; q < m; ++q) p = fmaf(-l[m][q], l[m][q], p);
    const bool real = 4 * K + m < n;
    ok = ok && (!real || p > tol);
    p = real ? p : 1.0f;
    rr[m] = rsqrtf(p);
    l[m][m] = p * rr[m];
#pragma unroll
    for (int i = m + 1; i < 4; ++i) {
      float s = d[i][m];
#pragma unroll
      for (int q = 0; q < m; ++q) s = fmaf(-l[i][q], l[m][q], s);
      l[i][m] = s * rr[m];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j > i) { w[i][j] = 0.0f; continue; }
      if (j == i) { w[i][j] = rr[i]; continue; }
      float s = 0.0f;
#pragma unroll
      for (int q = j; q < i; ++q) s = fmaf(l[i][q], w[q][j], s);
      w[i][j] = -rr[i] * s;
    }
  }
  return ok;
}

}  // namespace ci

// Every thread of the CTA calls this (blockDim.x >= chol_inv_threads(n), 4 <= n <= 128).
// On success W = L^-1 is written as the padded column-major image Wimg[c * (n + 1) + r]
// (zeros above the diagonal) and true is returned; when a pivot is <= tol_scale * max diag K
// nothing is written and false is returned (by every thread).
__device__ __forceinline__ bool chol_inv_tiles(int n, float tol_scale,
                                               const float* __restrict__ pre, int lda,
                                               float* __restrict__ Wimg, CiShared& s) {
  const int nb = (n + 3) >> 2;
  const int t = threadIdx.x;
  const bool act = t < nb * (nb + 1) / 2;
  int bi = 0;
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  const int bj = t - bi * (bi + 1) / 2;
  float a[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = 4 * bj + c;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act && col < n)
      x = *reinterpret_cast<const float4*>(pre + static_cast<int64_t>(col) * lda + 4 * bi);
    const float xr[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = 4 * bi + r;
      a[r][c] = (act && col < n && i < n && i >= col) ? xr[r] : 0.f;
    }
  }
  if (t < 32) {   // the largest diagonal entry: all loads issued before the first use
    float dv[kCiMaxN / 32];
#pragma unroll
    for (int q = 0; q < kCiMaxN / 32; ++q) {
      const int i = t + 32 * q;
      dv[q] = i < n ? pre[static_cast<int64_t>(i) * lda + i] : 0.f;
    }
    float md = 0.f;
#pragma unroll
    for (int q = 0; q < kCiMaxN / 32; ++q) md = fmaxf(md, dv[q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    if (t == 0) s.tol = tol_scale * md;
  }
  if (t < 4) s.Id[t] = make_float4(t == 0, t == 1, t == 2, t == 3);
  __syncthreads();
  const float tol = s.tol;
  if (act && bj == 0) ci::st(s.P[0][bi], a);
  if (t == 0) {
    float w0[4][4];
    s.ok[0] = ci::factor_block(a, 0, n, tol, w0) ? 1 : 0;
    ci::st(s.W[0], w0);
  }
  __syncthreads();
  for (int K = 0; K < nb; ++K) {
    const int b = K & 1;
    if (!s.ok[b]) return false;
    float w[4][4];
    ci::ld(s.W[b], w);
    if (act && bi == K) {                   // block row K: W_{K,bj} = W_KK R_{K,bj}
      float o[4][4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v = 0.f;
#pragma unroll
          for (int q = 0; q <= m; ++q) v = fmaf(w[m][q], bj == K ? (q == c ? 1.f : 0.f) : a[q][c], v);
          o[m][c] = v;
        }
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int c = 0; c < 4; ++c) a[m][c] = o[m][c];
    } else if (act && bi > K) {             // the update: tile -= L_{bi,K} Y
      float P[4][4], M[4][4], Li[4][4], Y[4][4];
      ci::ld(s.P[b][bi], P);
      ci::ld(bj > K ? s.P[b][bj] : (bj == K ? s.Id : s.R[b][bj]), M);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          float v = 0.f;
#pragma unroll
          for (int q = 0; q <= m; ++q) v = fmaf(P[r][q], w[m][q], v);
          Li[r][m] = v;
        }
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v = 0.f;
#pragma unroll
          for (int q = 0; q <= m; ++q) v = fmaf(w[m][q], M[c][q], v);
          Y[m][c] = v;
        }
      const bool fresh = bj == K;
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float v = fresh ? 0.f : a[r][c];
#pragma unroll
          for (int m = 0; m < 4; ++m) v = fmaf(-Li[r][m], Y[m][c], v);
          a[r][c] = v;
        }
    }
    const int K1 = K + 1;
    if (act && K1 < nb) {
      if (bj == K1) {
        ci::st(s.P[K1 & 1][bi], a);
        if (bi == K1) {
          float w1[4][4];
          s.ok[K1 & 1] = ci::factor_block(a, K1, n, tol, w1) ? 1 : 0;
          ci::st(s.W[K1 & 1], w1);
        }
      }
      if (bi == K1 && bj <= K) ci::st_t(s.R[K1 & 1][bj], a);
    }
    __syncthreads();
  }
  if (act) {
    const int np = n + 1;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = 4 * bi + r;
      if (i >= n) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = 4 * bj + c;
        if (col >= n) continue;
        Wimg[col * np + i] = i >= col ? a[r][c] : 0.f;
        if (bi != bj) Wimg[i * np + col] = 0.f;   // the mirrored tile above the diagonal
      }
    }
  }
  return true;
}

}  // namespace trk
