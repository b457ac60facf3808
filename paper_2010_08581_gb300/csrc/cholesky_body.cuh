// One-CTA Cholesky factorisation G = L L^T (n <= 256), shared by the single-problem kernel
// and the batched kernel. Used for the normal matrix of the sampled LS (row a6, Alg. 2 LS
// step) and for the R factor of the Cholesky-based thin QR behind the leverage scores
// (row a1).
//
// Right-looking with one column of look-ahead. At step k column k is final; warp 0 applies
// column k's update to column k+1 only, takes its pivot (rsqrt) and scales it, while warps
// 1.. apply column k's rank-1 update to the trailing triangle of columns >= k+2. One barrier
// per column. A is the n x n work array (shared memory, or global scratch).
//
// The working type T is double or float. In FP64 the trailing triangle's (m+1)m/2 entries
// are spread evenly over the threads (every lane busy: the FP64 pipe is the bound); every
// update is one fused multiply-add, a_ij = fma(-l_ik, l_jk, a_ij). In FP32 (the mixed-precision LS step, whose triangular solves already
// run in FP32) a warp takes whole rows and its lanes the columns, with no index arithmetic
// per entry.
//
// mode 0 (solve): a pivot <= tol_scale * max diag stops the factorisation (*info = column
// + 1, singular bit). mode 1 (leverage): such a column is dropped (zero, keep = 0).
// A non-final attempt (`final_attempt` false: the FP32 try of the mixed LS step) that stops
// writes nothing and returns false; its caller then factors in FP64.
// Besides L (row- and column-major, if Lrow/Lcol are given) the kernel can write padded
// images that the triangular-solve kernels copy straight into shared memory:
// img[c*(n+1) + r] = L[r][c] in FP64 and/or FP32, and the FP32 image of the symmetric input.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace trk {

constexpr int CNT = 512;

__device__ __forceinline__ double chol_rsqrt(double d) { return rsqrt(d); }
__device__ __forceinline__ float chol_rsqrt(float d) { return rsqrtf(d); }
__device__ __forceinline__ double chol_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float chol_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double chol_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float chol_max(float a, float b) { return fmaxf(a, b); }

template <typename T>
__device__ __forceinline__ bool cholesky_cta(const double* __restrict__ G, int n, int mode,
                                             double tol_scale, T* A, double* Lrow,
                                             double* Lcol, double* invdiag, int* keep_out,
                                             int* info, unsigned* err, double* img64,
                                             float* img32, float* gimg32,
                                             bool final_attempt = true) {
  __shared__ T colbuf[2][kMaxL];
  __shared__ int keepv[kMaxL];
  __shared__ T s_tol;
  __shared__ int s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = n + 1;
  for (int e = tid; e < n * n; e += CNT) {
    const int i = e / n, j = e - (e / n) * n;
    if (j <= i) {
      const double g = G[static_cast<int64_t>(j) * n + i];
      A[e] = static_cast<T>(g);
      if (gimg32) {
        gimg32[j * np + i] = static_cast<float>(g);
        gimg32[i * np + j] = static_cast<float>(g);
      }
    } else {
      A[e] = T(0);
    }
  }
  __syncthreads();
  if (warp == 0) {
    T md = T(0);
    for (int i = lane; i < n; i += 32) md = chol_max(md, A[i * n + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = chol_max(md, __shfl_xor_sync(0xffffffffu, md, o));
    const T tol = static_cast<T>(tol_scale) * md;
    const T d = A[0];
    const bool ok = d > tol;                  // false for NaN and non-positive pivots
    const T inv = ok ? chol_rsqrt(d) : T(0);
    for (int i = lane; i < n; i += 32) {
      const T v = ok ? ((i == 0) ? d * inv : A[i * n] * inv) : T(0);
      A[i * n] = v;
      colbuf[0][i] = v;
    }
    if (lane == 0) {
      s_tol = tol;
      keepv[0] = ok ? 1 : 0;
      s_stop = (!ok && mode == 0) ? 1 : 0;
    }
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (s_stop) break;
    const T* cur = colbuf[k & 1];
    T* nxt = colbuf[(k + 1) & 1];
    const bool kp = keepv[k] != 0;
    if (warp == 0) {
      if (k + 1 < n) {
        // column k+1: a_i = A[i][k+1] - L[i][k] L[k+1][k]; pivot; scale
        const T lk1 = cur[k + 1];
        T a[kMaxL / 32];
#pragma unroll
        for (int q = 0; q < kMaxL / 32; ++q) {
          const int i = k + 1 + lane + 32 * q;
          a[q] = T(0);
          if (i < n) a[q] = kp ? chol_fma(-cur[i], lk1, A[i * n + k + 1]) : A[i * n + k + 1];
        }
        const T d = __shfl_sync(0xffffffffu, a[0], 0);   // row k+1: lane 0, q = 0
        const bool ok = d > s_tol;
        const T inv = ok ? chol_rsqrt(d) : T(0);
#pragma unroll
        for (int q = 0; q < kMaxL / 32; ++q) {
          const int i = k + 1 + lane + 32 * q;
          if (i < n) {
            const T v = ok ? ((i == k + 1) ? d * inv : a[q] * inv) : T(0);
            A[i * n + k + 1] = v;
            nxt[i] = v;
          }
        }
        if (lane == 0) {
          keepv[k + 1] = ok ? 1 : 0;
          if (!ok && mode == 0) s_stop = k + 2;
        }
      }
    } else if (!kp) {
      // a dropped column updates nothing
    } else if constexpr (sizeof(T) == 4) {
      // trailing triangle, FP32: warp w takes rows k+2+(w-1), k+2+(w-1)+(W-1), ...; its
      // lanes the columns k+2 .. i of the row
      const int j0 = k + 2;
      for (int i = j0 + warp - 1; i < n; i += CNT / 32 - 1) {
        const T li = cur[i];
        T* row = A + i * n;
        for (int j = j0 + lane; j <= i; j += 32) row[j] = chol_fma(-li, cur[j], row[j]);
      }
    } else {
      // trailing triangle of columns >= k+2: rows i >= j >= k+2
      const int m = n - k - 2;
      const int P = m > 0 ? m * (m + 1) / 2 : 0;
      for (int e = tid - 32; e < P; e += CNT - 32) {
        int ii = static_cast<int>((sqrtf(8.0f * static_cast<float>(e) + 1.0f) - 1.0f) * 0.5f);
        while (ii * (ii + 1) / 2 > e) --ii;
        while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
        const int jj = e - ii * (ii + 1) / 2;
        const int i = k + 2 + ii, j = k + 2 + jj;
        A[i * n + j] = fma(-cur[i], cur[j], A[i * n + j]);
      }
    }
    __syncthreads();
  }
  const int stop = s_stop;
  if (stop && !final_attempt) return false;
  if (tid == 0) {
    *info = stop;
    if (stop) atomicOr(err, kErrSingular);
  }
  if (stop) return true;
  for (int e = tid; e < n * n; e += CNT) {
    const int i = e / n, j = e - (e / n) * n;
    const T v = (j <= i) ? A[e] : T(0);
    if (Lrow) Lrow[e] = static_cast<double>(v);
    if (Lcol) Lcol[static_cast<int64_t>(j) * n + i] = static_cast<double>(v);
    if (img64) img64[j * np + i] = static_cast<double>(v);
    if (img32) img32[j * np + i] = static_cast<float>(v);
  }
  for (int k = tid; k < n; k += CNT) {
    keep_out[k] = keepv[k];
    invdiag[k] = keepv[k] ? 1.0 / static_cast<double>(A[k * n + k]) : 0.0;
  }
  return true;
}

// Blocked right-looking Cholesky for n <= kPanelCholMax in a working arithmetic `Ops`:
// FP32 (F32Ops, the mixed LS step) or double-float (FFOps, a value hi + lo of two FP32
// numbers, about 46 significant bits: the mixed path's leverage Gram). Panels of Ops::kPB columns:
// warp 0 factors a panel in registers (lane l holds rows c0 + l + 32q of the panel's
// columns): per column one shuffle for the pivot, an rsqrt, a scaling and kPB-1 shuffles for
// the later panel columns, with no barrier. The panel's rank-kPB update is applied to 4 x 4
// tiles of the trailing lower triangle, reading the panel columns as 16-byte vectors from the
// column-major work array A (Ops::kPlanes planes of lda * n floats, lda a multiple of 4).
// With one panel of look-ahead: warp 0 updates and factors the next panel while the other
// warps update the rest, one barrier per panel. Every entry receives its updates in column
// order, so the factor does not depend on the schedule.
// The factor image img (FP32 or FP64, padded column-major) is written once at the end.
// Returns false (no factor written) when a pivot is <= tol_scale * max diag.
constexpr int kPanelCholMax = 160;

__host__ __device__ inline int panel_lda(int n) { return (n + 3) & ~3; }

struct F32Ops {
  using V = float;
  static constexpr int kPlanes = 1;
  static constexpr int kPB = 8;      // panel width
  __device__ static V from(double g) { return static_cast<float>(g); }
  __device__ static V zero() { return 0.0f; }
  __device__ static float lead(V v) { return v; }
  __device__ static double wide(V v) { return static_cast<double>(v); }
  __device__ static V fnms(V x, V y, V a) { return fmaf(-x, y, a); }   // a - x*y
  __device__ static V mul(V x, V y) { return x * y; }
  __device__ static V rsqrt(V d) { return rsqrtf(d); }
  __device__ static V shfl(V v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  __device__ static V ld(const float* A, int o, int) { return A[o]; }
  __device__ static void st(float* A, int o, int, V v) { A[o] = v; }
  __device__ static void ld4(const float* A, int o, int, V (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(A + o);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ static void st4(float* A, int o, int, const V (&v)[4]) {
    *reinterpret_cast<float4*>(A + o) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

// Double-float values (Dekker 1971; products via fused multiply-add). fnms: the exact product
// of the leading parts plus the cross terms, then a two-sum with the accumulator; rsqrt: the
// FP32 estimate refined by one Newton step with the residual formed in double-float.
struct ffv { float hi, lo; };
template <int PB>
struct FFOpsT {
  using V = ffv;
  static constexpr int kPlanes = 2;
  static constexpr int kPB = PB;     // panel width (registers: a double-float is two floats)
  __device__ static V from(double g) {
    const float h = static_cast<float>(g);
    return {h, static_cast<float>(g - static_cast<double>(h))};
  }
  __device__ static V zero() { return {0.0f, 0.0f}; }
  __device__ static float lead(V v) { return v.hi; }
  __device__ static double wide(V v) { return static_cast<double>(v.hi) + static_cast<double>(v.lo); }
  __device__ static V fnms(V x, V y, V a) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    const float s = a.hi - p;
    const float b = s - a.hi;
    float err = (a.hi - (s - b)) + (-p - b);
    err += a.lo - e;
    const float h = s + err;
    return {h, err - (h - s)};
  }
  __device__ static V mul(V x, V y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    const float h = p + e;
    return {h, e - (h - p)};
  }
  __device__ static V rsqrt(V d) {
    const float y0 = rsqrtf(d.hi);
    const float t = y0 * y0;
    const V tt{t, fmaf(y0, y0, -t)};               // y0^2 exactly
    const V dt = mul(d, tt);
    const float r = (1.0f - dt.hi) - dt.lo;        // 1 - d y0^2 (small)
    const float c = y0 * r * 0.5f;
    const float h = y0 + c;
    return {h, c - (h - y0)};
  }
  __device__ static V shfl(V v, int src) {
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
  }
  __device__ static V ld(const float* A, int o, int ps) { return {A[o], A[ps + o]}; }
  __device__ static void st(float* A, int o, int ps, V v) { A[o] = v.hi; A[ps + o] = v.lo; }
  __device__ static void ld4(const float* A, int o, int ps, V (&v)[4]) {
    const float4 h = *reinterpret_cast<const float4*>(A + o);
    const float4 l = *reinterpret_cast<const float4*>(A + ps + o);
    v[0] = {h.x, l.x}; v[1] = {h.y, l.y}; v[2] = {h.z, l.z}; v[3] = {h.w, l.w};
  }
  __device__ static void st4(float* A, int o, int ps, const V (&v)[4]) {
    *reinterpret_cast<float4*>(A + o) = make_float4(v[0].hi, v[1].hi, v[2].hi, v[3].hi);
    *reinterpret_cast<float4*>(A + ps + o) = make_float4(v[0].lo, v[1].lo, v[2].lo, v[3].lo);
  }
};

// 4-column panels: measured 107 us at n = 100 in the single-problem kernel, against 142 us
// with 8 (longer serial panel work in warp 0).
using FFOps = FFOpsT<4>;

// Floats of the work array of cholesky_panel<Ops>.
template <typename Ops>
__host__ __device__ inline int64_t panel_floats(int n) {
  return static_cast<int64_t>(Ops::kPlanes) * panel_lda(n) * n;
}

template <typename Ops, typename TI>
__device__ __forceinline__ bool cholesky_panel(const double* __restrict__ G, int n,
                                               double tol_scale, float* A, double* invdiag,
                                               int* keep_out, int* info, TI* img,
                                               float* gimg32, float* img_hi = nullptr,
                                               float* img_lo = nullptr,
                                               const float* pre_hi = nullptr,
                                               const float* pre_lo = nullptr) {
  using V = typename Ops::V;
  constexpr int QP = (kPanelCholMax + 31) / 32;
  constexpr int kPB = Ops::kPB;
  __shared__ V s_ldiag[kPanelCholMax];   // in the working type: converted once, at the end
  __shared__ float s_tol;
  __shared__ int s_stop;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NW = CNT / 32;
  const int np = n + 1, lda = panel_lda(n), ps = lda * n;
  // load: the lower triangle into A, the whole (symmetric) matrix into the FP32 image; each
  // thread issues the loads of two columns before any store. With pre_hi (pre_lo) the
  // reduction already wrote A's planes (and the FP32 image): a 16-byte copy.
  if (pre_hi) {
    const int tot = lda * n;                              // a multiple of 4
    for (int e = tid * 4; e < tot; e += CNT * 4) {
      *reinterpret_cast<float4*>(A + e) = *reinterpret_cast<const float4*>(pre_hi + e);
      if constexpr (Ops::kPlanes == 2)
        *reinterpret_cast<float4*>(A + ps + e) = *reinterpret_cast<const float4*>(pre_lo + e);
    }
  }
  for (int j0 = pre_hi ? n : warp; j0 < n; j0 += 2 * NW) {
    double g[2][QP];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < QP; ++q) {
        const int j = j0 + h * NW, i = lane + 32 * q;
        g[h][q] = (j < n && i < n) ? G[static_cast<int64_t>(j) * n + i] : 0.0;
      }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < QP; ++q) {
        const int j = j0 + h * NW, i = lane + 32 * q;
        if (j < n && i < n) {
          if (gimg32) gimg32[j * np + i] = static_cast<float>(g[h][q]);
          if (i >= j) Ops::st(A, j * lda + i, ps, Ops::from(g[h][q]));
        }
      }
  }
  if (warp == 0) {
    float dg[QP];
#pragma unroll
    for (int q = 0; q < QP; ++q) {
      const int i = lane + 32 * q;
      dg[q] = (i < n) ? (pre_hi ? pre_hi[i * lda + i]
                                : static_cast<float>(G[static_cast<int64_t>(i) * n + i]))
                      : 0.0f;
    }
    float md = 0.0f;
#pragma unroll
    for (int q = 0; q < QP; ++q) md = fmaxf(md, dg[q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    if (lane == 0) {
      s_tol = static_cast<float>(tol_scale) * md;
      s_stop = 0;
    }
  }
  __syncthreads();
  // Panel factorisation of columns [c0, c0 + w) by warp 0, in registers (lane l holds rows
  // c0 + l + 32q, q < QPD, of the panel's columns): per column one shuffle for the pivot, an
  // rsqrt, a scaling and w - 1 shuffles for the later panel columns, with no barrier. QPD is
  // the number of 32-row slots the panel's rows need (instantiated per count).
  auto factor_panel_q = [&](auto qc, int c0) {
    constexpr int QPD = decltype(qc)::value;
    const int w = (n - c0 < kPB) ? n - c0 : kPB;
    V p[QPD][kPB];
#pragma unroll
    for (int q = 0; q < QPD; ++q) {
      const int i = c0 + lane + 32 * q;
#pragma unroll
      for (int jj = 0; jj < kPB; ++jj)
        p[q][jj] = (i < n && jj < w && i >= c0 + jj) ? Ops::ld(A, (c0 + jj) * lda + i, ps)
                                                     : Ops::zero();
    }
    const float tol = s_tol;
    bool ok = true;
#pragma unroll
    for (int kk = 0; kk < kPB; ++kk) {
      if (kk < w) {
        const V d = Ops::shfl(p[0][kk], kk);                       // row c0+kk: lane kk
        ok = ok && (Ops::lead(d) > tol);
        const V inv = ok ? Ops::rsqrt(d) : Ops::zero();
#pragma unroll
        for (int q = 0; q < QPD; ++q) {
          const int r = lane + 32 * q;                              // panel row
          p[q][kk] = (r == kk) ? Ops::mul(d, inv)
                               : (r > kk ? Ops::mul(p[q][kk], inv) : Ops::zero());
        }
#pragma unroll
        for (int jj = kk + 1; jj < kPB; ++jj) {
          const V ljk = Ops::shfl(p[0][kk], jj);                    // row c0+jj: lane jj
#pragma unroll
          for (int q = 0; q < QPD; ++q) p[q][jj] = Ops::fnms(p[q][kk], ljk, p[q][jj]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < QPD; ++q) {
      const int i = c0 + lane + 32 * q;
      if (i < n) {
#pragma unroll
        for (int jj = 0; jj < kPB; ++jj)
          if (jj < w && i >= c0 + jj) {
            Ops::st(A, (c0 + jj) * lda + i, ps, p[q][jj]);
            if (i == c0 + jj) s_ldiag[i] = p[q][jj];
          }
      }
    }
    if (lane == 0 && !ok) s_stop = 1;
  };
  auto factor_panel = [&](int c0) {
    const int slots = (n - c0 + 31) >> 5;
    if (slots <= 1) factor_panel_q(std::integral_constant<int, 1>{}, c0);
    else if (slots == 2) factor_panel_q(std::integral_constant<int, 2>{}, c0);
    else if (slots == 3) factor_panel_q(std::integral_constant<int, 3>{}, c0);
    else if (slots == 4) factor_panel_q(std::integral_constant<int, 4>{}, c0);
    else factor_panel_q(std::integral_constant<int, QP>{}, c0);
  };
  // Rank-w update of the 4 x 4 tile (bi, bj) of the trailing triangle at t0 with the panel
  // [c0, c0 + w): every entry receives the panel's columns in order.
  auto update_tile = [&](int c0, int w, int t0, int bi, int bj) {
    const int i0 = t0 + 4 * bi, j0 = t0 + 4 * bj;
    V acc[4][4];   // acc[c][r]: column j0+c, row i0+r
#pragma unroll
    for (int c = 0; c < 4; ++c) {   // columns >= n do not exist (rows up to lda do)
      if (j0 + c < n) {
        Ops::ld4(A, (j0 + c) * lda + i0, ps, acc[c]);
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = Ops::zero();
      }
    }
#pragma unroll
    for (int kk = 0; kk < kPB; ++kk) {
      if (kk < w) {
        V li[4], lj[4];
        Ops::ld4(A, (c0 + kk) * lda + i0, ps, li);
        Ops::ld4(A, (c0 + kk) * lda + j0, ps, lj);
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[c][r] = Ops::fnms(li[r], lj[c], acc[c][r]);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (j0 + c < n) Ops::st4(A, (j0 + c) * lda + i0, ps, acc[c]);
  };
  // One panel of look-ahead. After panel c0 is final (barrier), warp 0 applies it to the next
  // panel's columns (tile columns bj < kPB / 4 of the trailing triangle) and factors that panel,
  // while the other warps apply panel c0 to the rest of the trailing triangle. One barrier per
  // panel; the next panel's factorisation overlaps the trailing update.
  if (warp == 0) factor_panel(0);
  __syncthreads();
  if (s_stop) return false;
  constexpr int PB4 = kPB / 4;                      // tile columns of one panel
  for (int c0 = 0; c0 < n; c0 += kPB) {
    const int w = (n - c0 < kPB) ? n - c0 : kPB;
    const int t0 = c0 + w;
    const int m = n - t0;
    if (m > 0) {
      const int nb = (m + 3) >> 2;
      const int pb = nb < PB4 ? nb : PB4;
      if (warp == 0) {
        for (int bj = 0; bj < pb; ++bj)
          for (int bi = bj + lane; bi < nb; bi += 32) update_tile(c0, w, t0, bi, bj);
        __syncwarp();
        factor_panel(t0);
      } else {
        // tiles with bj >= pb: the triangle of size nb - pb starting at (pb, pb)
        const int mb = nb - pb;
        const int ntiles = mb * (mb + 1) / 2;
        for (int t = tid - 32; t < ntiles; t += CNT - 32) {
          int bi = static_cast<int>((sqrtf(8.0f * static_cast<float>(t) + 1.0f) - 1.0f) * 0.5f);
          while (bi * (bi + 1) / 2 > t) --bi;
          while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
          const int bj = t - bi * (bi + 1) / 2;
          update_tile(c0, w, t0, bi + pb, bj + pb);
        }
      }
    }
    __syncthreads();
    if (s_stop) return false;
  }
  // the factor image, padded column-major: img[c*(n+1) + r] = L[r][c]; or, for a
  // double-float factor with img_hi/img_lo given, its two FP32 planes in that layout (the
  // FP64 image is then formed by launch_ff_image, across many SMs: *info = 2 marks it)
  if constexpr (Ops::kPlanes == 2) {
    if (img_hi) {
      for (int j = warp; j < n; j += NW)
        for (int i = lane; i < n; i += 32) {
          const V v = (i >= j) ? Ops::ld(A, j * lda + i, ps) : Ops::zero();
          img_hi[j * np + i] = Ops::lead(v);
          img_lo[j * np + i] = v.lo;
        }
    }
  }
  if (!img_hi)
    for (int j = warp; j < n; j += NW)
      for (int i = lane; i < n; i += 32)
        img[j * np + i] =
            (i >= j) ? static_cast<TI>(Ops::wide(Ops::ld(A, j * lda + i, ps))) : TI(0);
  for (int k = tid; k < n; k += CNT) {
    keep_out[k] = 1;
    invdiag[k] = 1.0 / Ops::wide(s_ldiag[k]);
  }
  if (tid == 0) *info = img_hi ? 2 : 0;
  return true;
}

// Blocked right-looking FP32 Cholesky without look-ahead, for any block size (blockDim.x a
// multiple of 32, at least 64): per panel of kP32 columns, warp 0 factors the panel in
// registers (as cholesky_panel, with QPD 32-row slots sized to the rows left), one barrier,
// then every thread takes 4 x 4 tiles of the rank-kP32 update of the trailing triangle, one
// barrier. At n = 100 this measured 31 us with 256 threads against 39 us for cholesky_panel
// with one panel of look-ahead and 512 threads: the look-ahead kept warp 0 busy with tile
// updates on the critical path, and a 512-thread barrier costs more. A: the work array (as
// cholesky_panel, FP32, lda = panel_lda(n)), filled from pre (the reduction's FP32 work array).
// Writes the padded factor image img (FP32), invdiag (FP64), keep (all 1) and *info = 0;
// returns false (nothing written) when a pivot is <= tol_scale * max diag.
constexpr int kP32 = 8;

template <int QPD>
__device__ __forceinline__ bool factor_panel_p32(float* A, int lda, int n, int c0, float tol,
                                                 float* ldiag) {
  const int lane = threadIdx.x & 31;
  const int w = (n - c0 < kP32) ? n - c0 : kP32;
  float p[QPD][kP32];
#pragma unroll
  for (int q = 0; q < QPD; ++q) {
    const int i = c0 + lane + 32 * q;
#pragma unroll
    for (int jj = 0; jj < kP32; ++jj)
      p[q][jj] = (i < n && jj < w && i >= c0 + jj) ? A[(c0 + jj) * lda + i] : 0.f;
  }
  bool ok = true;
#pragma unroll
  for (int kk = 0; kk < kP32; ++kk) {
    if (kk < w) {
      const float d = __shfl_sync(0xffffffffu, p[0][kk], kk);
      ok = ok && (d > tol);
      const float inv = ok ? rsqrtf(d) : 0.f;
#pragma unroll
      for (int q = 0; q < QPD; ++q) {
        const int r = lane + 32 * q;
        p[q][kk] = (r == kk) ? d * inv : (r > kk ? p[q][kk] * inv : 0.f);
      }
#pragma unroll
      for (int jj = kk + 1; jj < kP32; ++jj) {
        const float ljk = __shfl_sync(0xffffffffu, p[0][kk], jj);
#pragma unroll
        for (int q = 0; q < QPD; ++q) p[q][jj] = fmaf(-p[q][kk], ljk, p[q][jj]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QPD; ++q) {
    const int i = c0 + lane + 32 * q;
#pragma unroll
    for (int jj = 0; jj < kP32; ++jj)
      if (i < n && jj < w && i >= c0 + jj) {
        A[(c0 + jj) * lda + i] = p[q][jj];
        if (i == c0 + jj) ldiag[i] = p[q][jj];
      }
  }
  return ok;
}

__device__ __forceinline__ bool cholesky_panel_f32(int n, double tol_scale, float* A,
                                                   const float* __restrict__ pre, float* img,
                                                   double* invdiag, int* keep_out, int* info) {
  __shared__ float ldiag[kPanelCholMax];
  __shared__ float s_tol;
  __shared__ int s_bad;
  const int nt = blockDim.x;
  const int lda = panel_lda(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid * 4; e < lda * n; e += nt * 4)
    *reinterpret_cast<float4*>(A + e) = *reinterpret_cast<const float4*>(pre + e);
  if (warp == 0) {
    float md = 0.f;
    for (int i = lane; i < n; i += 32) md = fmaxf(md, pre[i * lda + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    if (lane == 0) {
      s_tol = static_cast<float>(tol_scale) * md;
      s_bad = 0;
    }
  }
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += kP32) {
    if (warp == 0) {
      const int slots = (n - c0 + 31) >> 5;
      bool ok;
      if (slots <= 1) ok = factor_panel_p32<1>(A, lda, n, c0, s_tol, ldiag);
      else if (slots == 2) ok = factor_panel_p32<2>(A, lda, n, c0, s_tol, ldiag);
      else if (slots == 3) ok = factor_panel_p32<3>(A, lda, n, c0, s_tol, ldiag);
      else if (slots == 4) ok = factor_panel_p32<4>(A, lda, n, c0, s_tol, ldiag);
      else ok = factor_panel_p32<(kPanelCholMax + 31) / 32>(A, lda, n, c0, s_tol, ldiag);
      if (!ok && lane == 0) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) return false;
    // rank-w update of the trailing triangle (rows i >= j >= t0), 4 x 4 tiles; rows up to
    // lda exist in every column (lda = panel_lda(n)), columns >= n are skipped
    const int w = (n - c0 < kP32) ? n - c0 : kP32;
    const int t0 = c0 + w, m = n - t0;
    if (m > 0) {
      const int nb = (m + 3) >> 2;
      const int ntiles = nb * (nb + 1) / 2;
      for (int t = tid; t < ntiles; t += nt) {
        int bi = static_cast<int>((sqrtf(8.0f * static_cast<float>(t) + 1.0f) - 1.0f) * 0.5f);
        while (bi * (bi + 1) / 2 > t) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        const int bj = t - bi * (bi + 1) / 2;
        const int i0 = t0 + 4 * bi, j0 = t0 + 4 * bj;
        float acc[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (j0 + c < n) {
            const float4 v = *reinterpret_cast<const float4*>(A + (j0 + c) * lda + i0);
            acc[c][0] = v.x; acc[c][1] = v.y; acc[c][2] = v.z; acc[c][3] = v.w;
          } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[c][r] = 0.f;
          }
        }
#pragma unroll
        for (int kk = 0; kk < kP32; ++kk) {
          if (kk < w) {
            const float4 li = *reinterpret_cast<const float4*>(A + (c0 + kk) * lda + i0);
            const float4 lj = *reinterpret_cast<const float4*>(A + (c0 + kk) * lda + j0);
            const float a4[4] = {li.x, li.y, li.z, li.w}, b4[4] = {lj.x, lj.y, lj.z, lj.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int r = 0; r < 4; ++r) acc[c][r] = fmaf(-a4[r], b4[c], acc[c][r]);
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (j0 + c < n)
            *reinterpret_cast<float4*>(A + (j0 + c) * lda + i0) =
                make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
      }
    }
    __syncthreads();
  }
  const int np = n + 1;
  for (int j = warp; j < n; j += nt / 32)
    for (int i = lane; i < n; i += 32) img[j * np + i] = (i >= j) ? A[j * lda + i] : 0.f;
  for (int k = tid; k < n; k += nt) {
    keep_out[k] = 1;
    invdiag[k] = 1.0 / static_cast<double>(ldiag[k]);
  }
  if (tid == 0) *info = 0;
  return true;
}

// FP32 first, FP64 if needed: the factorisation of the mixed-precision LS step's normal
// matrix (mode 0, image TI = float). The FP32 attempt accepts the factor only if every pivot
// exceeds tol32 * max diag (so it never drops a column); otherwise the same matrix is factored
// in FP64 with the mode's rule: mode 0 stops at tol64, mode 1 drops columns at tol32 (the
// resolution of the FP32 solves that follow). A32 and A64 are the work arrays (they may alias).
// Lrow/Lcol receive the FP64 factor only on the FP64 branch. (The sampling distributions keep
// their FP64 factorisation: FP32 rounding in p would change which indices the inverse CDF
// draws.)
template <typename TI>
__device__ __forceinline__ void cholesky_cta_mixed(const double* __restrict__ G, int n, int mode,
                                                   double tol64, double tol32, float* A32,
                                                   double* A64, double* Lrow, double* Lcol,
                                                   double* invdiag, int* keep_out, int* info,
                                                   unsigned* err, TI* img, float* gimg32,
                                                   const float* pre = nullptr) {
  constexpr bool f32img = sizeof(TI) == 4;
  double* img64 = f32img ? nullptr : reinterpret_cast<double*>(img);
  float* img32 = f32img ? reinterpret_cast<float*>(img) : nullptr;
  if (n >= 4 && n <= kPanelCholMax && img && pre && f32img) {   // (gimg32: written by the reduction)
    if (cholesky_panel_f32(n, tol32, A32, pre, reinterpret_cast<float*>(img), invdiag,
                           keep_out, info))
      return;
  } else if (n >= 4 && n <= kPanelCholMax && img) {
    if (cholesky_panel<F32Ops, TI>(G, n, tol32, A32, invdiag, keep_out, info, img, gimg32,
                                   nullptr, nullptr, pre))
      return;
  } else if (cholesky_cta<float>(G, n, 0, tol32, A32, nullptr, nullptr, invdiag, keep_out,
                                 info, err, img64, img32, gimg32, false)) {
    return;
  }
  __syncthreads();
  // Dropping (mode 1) keeps only columns the FP32 triangular solves can resolve: the FP32
  // tolerance. Stopping (mode 0) applies the FP64 rule.
  cholesky_cta<double>(G, n, mode, mode == 1 ? tol32 : tol64, A64, Lrow, Lcol, invdiag,
                       keep_out, info, err, img64, img32, gimg32, true);
}

// The mixed-precision drivers' leverage Gram of a tall matrix (mode 1): double-float first
// (panel width PB),
// accepted only if every pivot exceeds tolff * max diag (no column is dropped); otherwise
// the FP64 factorisation with tol64 and mode 1's column dropping. The image is FP64.
// Aff is the double-float work array (panel_floats<FFOps>(n) floats), A64 the FP64 one (they
// may alias). Lrow/Lcol receive the factor only on the FP64 branch; on the double-float
// branch they hold the image's hi / lo FP32 planes, *info = 2, and launch_ff_image (or the
// batched kb_ff_image) forms img64 from them.
template <int PB = 4>
__device__ __forceinline__ void cholesky_cta_lev_mixed(const double* __restrict__ G, int n,
                                                       double tol64, double tolff, float* Aff,
                                                       double* A64, double* Lrow, double* Lcol,
                                                       double* invdiag, int* keep_out,
                                                       int* info, unsigned* err, double* img64,
                                                       const float* pre_hi = nullptr,
                                                       const float* pre_lo = nullptr) {
  if (n >= 4 && n <= kPanelCholMax && img64 && Aff) {
    if (cholesky_panel<FFOpsT<PB>, double>(G, n, tolff, Aff, invdiag, keep_out, info, img64, nullptr,
                                      reinterpret_cast<float*>(Lrow),
                                      reinterpret_cast<float*>(Lcol), pre_hi, pre_lo))
      return;
    __syncthreads();
  }
  cholesky_cta<double>(G, n, 1, tol64, A64, Lrow, Lcol, invdiag, keep_out, info, err, img64,
                       nullptr, nullptr, true);
}

}  // namespace trk
