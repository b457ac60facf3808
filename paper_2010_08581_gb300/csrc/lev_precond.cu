// Row a1 in the mixed-precision drivers: the leverage scores of a tall I x n matrix A (Def. 4,
// the equation for p^(n)), ell_i = a_i^T K^-1 a_i with K = A^T A, through an FP32
// preconditioner instead of a double-float factorisation of K.
//
// For any nonsingular X, K^-1 = X^T (X K X^T)^-1 X, so with w_i = X a_i and C = X K X^T,
//   ell_i = w_i^T C^-1 w_i.
// X = L^-1 from the FP32 Cholesky factor of K (factor and inverse in one CTA, k_chol_inv)
// makes C = I + E with E small (of order n * eps32 * cond(K)). Then
//   C^-1 = I - E + E^2 - ...,   ell_i = w.w - w.v1 + v1.v1 - v1.v2 + v2.v2 - v2.v3 + v3.v3 - ...
// with v1 = E w, v2 = E v1, v3 = E v2. X only has to be a good preconditioner: C and w are
// formed from the same X, so the identity holds for the X actually computed. The products
// that carry the leading digits (C = X K X^T, w = X a, w.w) run in double-float (hi + lo FP32
// pairs, compensated dot products after Ogita, Rump and Oishi, SIAM J. Sci. Comput. 2005);
// E is then rounded to FP32 and the corrections, which are smaller than ell_i by the factor
// ||E||, run in FP32. All of this is parallel work over many CTAs; the only serial chain
// is the one-CTA pass that forms the FP32 factor and its inverse.
//
// The fast form is taken only when the FP32 factorisation succeeds (every pivot above
// n * eps32 * max diag) and ||E||_F <= tau (1e-2); the series then stops at E^2 (||E||_F <= 1e-5),
// E^4 (<= 1e-3) or E^6, leaving a truncation error below 1e-14 relative. The Gram K comes
// from one launch (k_gram_dd) in double-float. Otherwise the device flag
// `state` is set and the double-float factorisation with FP64 fallback (the rank rule of the
// FP64 path) runs instead, gated on the same flag, so both outcomes are decided on the device
// without a host round trip.
#include "chol_inv.cuh"
#include "cholesky_body.cuh"
#include "trsm_body.cuh"

namespace trk {

namespace {

constexpr float kTauF4 = 1e-3f;        // up to this, terms through E^4 suffice
constexpr int LT = 16;                 // tile edge of the products U = X K and C = U X^T
constexpr int kMaxPre = 128;           // largest n of the preconditioned form

__host__ __device__ inline int pad4(int v) { return (v + 3) & ~3; }

__device__ __forceinline__ void stage16(void* dst, const void* src, int bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const char* s = static_cast<const char*>(src);
  for (int o = threadIdx.x * 16; o < bytes; o += blockDim.x * 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d + o), "l"(s + o) : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

// Knuth's two-sum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Compensated accumulation (s, c) += x * (yh + yl): the product x*yh split exactly by a fused
// multiply-add, its leading part added by two-sum, the error terms gathered in c.
__device__ __forceinline__ void dot2_add(float& s, float& c, float x, float yh, float yl) {
  const float p = x * yh;
  const float pe = fmaf(x, yh, -p);
  float t, q;
  two_sum(s, p, t, q);
  s = t;
  c += q + fmaf(x, yl, pe);
}

// (s, c) -> normalised double-float (h, l), h = fl(s + c).
__device__ __forceinline__ void renorm(float s, float c, float& h, float& l) {
  h = s + c;
  l = c - (h - s);
}

// K = A^T A of a tall I x n matrix given as double-float planes, in one launch: CTA (tile,
// split) forms the split's 32 x 32 tile sum in compensated FP32 (each product's leading part
// and its exact error by a fused multiply-add, plus the cross terms, then a two-sum), writes
// it as an FP32 pair, and the CTA that finishes a tile last adds the splits' pairs in split
// order by two-sums. It writes K's double-float planes in the reduction's work-array layout
// (kh/kl[r*lda + c], c >= r) and K in FP64 (k64[r*n + c]) for the factorisation fallback.
constexpr int GD = 32, GDK = 32, GDNT = 256;
constexpr int kGramDdMaxSplits = 8;   // gram_dd_splits gives at most 8

__global__ void __launch_bounds__(GDNT) k_gram_dd(const float* __restrict__ Ah,
                                                  const float* __restrict__ Al, int64_t K, int n,
                                                  int64_t lda_a, int64_t chunk, int splits,
                                                  float* __restrict__ ph, float* __restrict__ pl,
                                                  unsigned* __restrict__ cnt,
                                                  float* __restrict__ kh, float* __restrict__ kl,
                                                  int lda, double* __restrict__ k64) {
  __shared__ float Ph[GDK][GD + 1], Pl[GDK][GD + 1];
  __shared__ float Qh[GDK][GD + 1], Ql[GDK][GD + 1];
  __shared__ int s_last;
  const int nt = (n + GD - 1) / GD;
  int tp = 0, rem = blockIdx.x;
  while (rem >= nt - tp) { rem -= nt - tp; ++tp; }
  const int tq = tp + rem;
  const int p0 = tp * GD, q0 = tq * GD;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * chunk;
  const int64_t k1 = (k0 + chunk < K) ? k0 + chunk : K;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  float sum[4] = {0.f, 0.f, 0.f, 0.f}, cor[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t kb = k0; kb < k1; kb += GDK) {
#pragma unroll
    for (int r = 0; r < (GDK * GD) / GDNT; ++r) {
      const int e = threadIdx.x + r * GDNT;
      const int kk = e / GD, col = e % GD;
      const int64_t t = kb + kk;
      const int p = p0 + col, q = q0 + col;
      const bool okp = t < k1 && p < n, okq = t < k1 && q < n;
      Ph[kk][col] = okp ? Ah[t * lda_a + p] : 0.f;
      Pl[kk][col] = okp ? Al[t * lda_a + p] : 0.f;
      Qh[kk][col] = okq ? Ah[t * lda_a + q] : 0.f;
      Ql[kk][col] = okq ? Al[t * lda_a + q] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GDK; ++kk) {
      const float yh = Qh[kk][tx], yl = Ql[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float xh = Ph[kk][ty + 8 * u], xl = Pl[kk][ty + 8 * u];
        const float pr = xh * yh;
        float er = fmaf(xh, yh, -pr);
        er = fmaf(xh, yl, er);
        er = fmaf(xl, yh, er);
        float t2, ts;
        two_sum(sum[u], pr, t2, ts);
        sum[u] = t2;
        cor[u] += ts + er;
      }
    }
    __syncthreads();
  }
  // this split's tile as FP32 pairs: [split][tile][32 x 32]
  const int64_t tb = (static_cast<int64_t>(blockIdx.y) * gridDim.x + blockIdx.x) * GD * GD;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = (ty + 8 * u) * GD + tx;
    ph[tb + e] = sum[u];
    pl[tb + e] = cor[u];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    s_last = (atomicAdd(cnt + blockIdx.x, 1u) == static_cast<unsigned>(splits) - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = (ty + 8 * u) * GD + tx;
    float hs = 0.f, hc = 0.f;
    for (int sp0 = 0; sp0 < splits; sp0 += kGramDdMaxSplits) {
      float vh[kGramDdMaxSplits], vl[kGramDdMaxSplits];   // all loads first, then the sums
#pragma unroll
      for (int k = 0; k < kGramDdMaxSplits; ++k) {
        const int sp = sp0 + k;
        const int64_t o = (static_cast<int64_t>(sp) * gridDim.x + blockIdx.x) * GD * GD + e;
        vh[k] = sp < splits ? __ldcg(ph + o) : 0.f;
        vl[k] = sp < splits ? __ldcg(pl + o) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < kGramDdMaxSplits; ++k) {
        float t2, ts;
        two_sum(hs, vh[k], t2, ts);
        hs = t2;
        hc += vl[k] + ts;
      }
    }
    float h, l;
    renorm(hs, hc, h, l);
    const int p = p0 + ty + 8 * u, q = q0 + tx;
    if (p < n && q < n) {
      k64[static_cast<int64_t>(p) * n + q] = static_cast<double>(h) + static_cast<double>(l);
      if (q >= p) {
        kh[p * lda + q] = h;
        kl[p * lda + q] = l;
      }
    }
  }
  if (threadIdx.x == 0) cnt[blockIdx.x] = 0u;
}

// The preconditioner X = L^-1 of K = L L^T in FP32, factor and inverse in one CTA
// (chol_inv_tiles). K comes from the reduction's FP32 work array. On success: the padded
// column-major image of X and *state = 0; when a pivot is <= tol_scale * max diag K:
// *state = 1 and nothing else.
__global__ void __launch_bounds__(kCiMaxThreads) k_chol_inv(int n, float tol_scale,
                                                            const float* __restrict__ pre,
                                                            int lda, float* __restrict__ Ximg,
                                                            int* __restrict__ state) {
  __shared__ CiShared cs;
  const bool ok = chol_inv_tiles(n, tol_scale, pre, lda, Ximg, cs);
  if (threadIdx.x == 0) *state = ok ? 0 : 1;
}

// The symmetric K[k][c] from its double-float planes, which hold the entries c >= r of row r
// (row stride lda).
__device__ __forceinline__ int ksym(int k, int c, int lda) {
  return k <= c ? k * lda + c : c * lda + k;
}

// U = X K in double-float, one 16 x 16 tile of U per CTA (thread (ty, tx): row i0 + ty,
// column c0 + tx): U_ic = sum_{k <= i} X[i][k] K[k][c], X lower triangular from the
// inverse's padded image (X[r][c] = Ximg[c*(n+1) + r]). Out: planes Uh, Ul, row stride ldu.
__global__ void __launch_bounds__(LT * LT) k_lev_u(int n, const float* __restrict__ Kh,
                                                   const float* __restrict__ Kl, int lda,
                                                   const float* __restrict__ Ximg,
                                                   const int* __restrict__ state,
                                                   float* __restrict__ Uh,
                                                   float* __restrict__ Ul, int ldu) {
  __shared__ float Xt[kMaxPre][LT + 1];        // X[i0 + r][k] at Xt[k][r]
  __shared__ float Kth[kMaxPre][LT], Ktl[kMaxPre][LT];
  if (*state != 0) return;
  const int np = n + 1;
  const int i0 = blockIdx.y * LT, c0 = blockIdx.x * LT;
  const int kmax = min(n, i0 + LT);
  const int t = threadIdx.y * LT + threadIdx.x;
  for (int e = t; e < kmax * LT; e += LT * LT) {
    const int k = e / LT, r = e - k * LT;
    const int i = i0 + r, c = c0 + r;
    Xt[k][r] = (i < n && k <= i) ? Ximg[k * np + i] : 0.f;
    const int o = ksym(k, c < n ? c : 0, lda);
    Kth[k][r] = c < n ? Kh[o] : 0.f;
    Ktl[k][r] = c < n ? Kl[o] : 0.f;
  }
  __syncthreads();
  const int i = i0 + threadIdx.y, c = c0 + threadIdx.x;
  if (i >= n || c >= n) return;
  float s = 0.f, cc = 0.f;
#pragma unroll 4
  for (int k = 0; k <= i; ++k) dot2_add(s, cc, Xt[k][threadIdx.y], Kth[k][threadIdx.x], Ktl[k][threadIdx.x]);
  float h, l;
  renorm(s, cc, h, l);
  Uh[i * ldu + c] = h;
  Ul[i * ldu + c] = l;
}

// E = U X^T - I = X K X^T - I on the tiles (ti, tj), ti <= tj, of the upper triangle, both
// triangles written (row stride lde, FP32), and the tile's share of ||E||_F^2 in esq[tile]:
// C_ij = sum_{k <= j} U[i][k] X[j][k] in double-float.
__global__ void __launch_bounds__(LT * LT) k_lev_e(int n, const float* __restrict__ Uh,
                                                   const float* __restrict__ Ul, int ldu,
                                                   const float* __restrict__ Ximg,
                                                   const int* __restrict__ state,
                                                   float* __restrict__ E, int lde,
                                                   float* __restrict__ esq) {
  __shared__ float Uth[LT][kMaxPre + 1], Utl[LT][kMaxPre + 1];   // U[i0 + r][k]
  __shared__ float Xt[kMaxPre][LT + 1];                          // X[j0 + r][k] at Xt[k][r]
  __shared__ float red[LT * LT / 32];
  if (*state != 0) return;
  const int np = n + 1;
  const int nt = (n + LT - 1) / LT;
  int ti = 0, rem = blockIdx.x;
  while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
  const int tj = ti + rem;
  const int i0 = ti * LT, j0 = tj * LT;
  const int kmax = min(n, j0 + LT);
  const int t = threadIdx.y * LT + threadIdx.x;
  for (int e = t; e < kmax * LT; e += LT * LT) {     // U rows: consecutive threads along k
    const int r = e / kmax, k = e - r * kmax;
    const int i = i0 + r;
    Uth[r][k] = i < n ? Uh[i * ldu + k] : 0.f;
    Utl[r][k] = i < n ? Ul[i * ldu + k] : 0.f;
  }
  for (int e = t; e < kmax * LT; e += LT * LT) {     // X rows: consecutive threads along j
    const int k = e / LT, r = e - k * LT;
    const int j = j0 + r;
    Xt[k][r] = (j < n && k <= j) ? Ximg[k * np + j] : 0.f;
  }
  __syncthreads();
  const int i = i0 + threadIdx.y, j = j0 + threadIdx.x;
  float sq = 0.f;
  if (i < n && j < n && i <= j) {
    float s = 0.f, cc = 0.f;
#pragma unroll 4
    for (int k = 0; k <= j; ++k)
      dot2_add(s, cc, Xt[k][threadIdx.x], Uth[threadIdx.y][k], Utl[threadIdx.y][k]);
    if (i == j) s -= 1.0f;          // exact when s is near 1 (Sterbenz)
    const float v = s + cc;
    E[i * lde + j] = v;
    E[j * lde + i] = v;
    sq = (i == j ? 1.0f : 2.0f) * v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((t & 31) == 0) red[t >> 5] = sq;
  __syncthreads();
  if (t == 0) {
    float a = 0.f;
    for (int w = 0; w < LT * LT / 32; ++w) a += red[w];
    esq[blockIdx.x] = a;
  }
}

// Warp sum of a double-float pair, the same butterfly in every lane.
__device__ __forceinline__ void warp_sum2(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    float t, q;
    two_sum(s, s2, t, q);
    s = t;
    c += c2 + q;
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int LR_ROWS = 4;             // rows of A per CTA of k_lev_rows
constexpr int LR_KS = 4;               // k-range split of w = X a
constexpr int LR_NT = 512;

// LR_ROWS rows of A per CTA: w = X a in double-float, ell = w.w - w.v1 + v1.v1 - ..., then
// (last CTA) p and the CDF. Every CTA reads the same ||E||_F^2 (fixed-order sum of esq); when
// it exceeds tau^2 no CTA computes anything and CTA 0 sets *state = 1 for the fallback.
// The series is cut where the next term is below 1e-15 relative: through E^2 for
// ||E||_F <= 1e-5, E^4 for <= 1e-3, E^6 otherwise.
// w: thread t serves rows 2h, 2h+1 (h = t / 64 % 2), the columns u and n-1-u (u = t % 64),
// which together take n+1 terms whatever u is (X is lower triangular), and a quarter of their
// k range (t / 128): four independent compensated chains; the quarters are then added in a
// fixed order. Products by E: thread t serves row t / 128 and column t % 128. X and E are
// staged in shared memory.
__global__ void __launch_bounds__(LR_NT) k_lev_rows(int n, int64_t I, const float* __restrict__ Ah,
                                                    const float* __restrict__ Al, int64_t lda,
                                                    const float* __restrict__ Ximg,
                                                    const float* __restrict__ E, int lde,
                                                    const float* __restrict__ esq, int nesq,
                                                    int* state, double* __restrict__ ell,
                                                    CdfEpilogue ep, float tau) {
  extern __shared__ __align__(16) float lrs[];  // X image, then E (row stride lde)
  __shared__ float2 as[LR_ROWS][kMaxPre];     // (a_hi, a_lo)
  __shared__ float wv[LR_ROWS][kMaxPre];      // w (FP32), then v1, v2
  __shared__ float part[LR_KS][128][8];       // quarter sums: (s, c) per row-column pair
  __shared__ float red[LR_NT / 32][8];
  if (*reinterpret_cast<volatile int*>(state) != 0) return;   // the FP32 factor failed
  float f2 = 0.f;
  for (int b = 0; b < nesq; ++b) f2 += esq[b];
  if (!(f2 <= tau * tau)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *state = 1;
    return;
  }
  const int nmv = f2 <= 1e-10f ? 1 : (f2 <= kTauF4 * kTauF4 ? 2 : 3);   // products by E
  const int np = n + 1;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int xi = pad4(n * np);
  float* Xs = lrs;
  float* Es = lrs + xi;
  stage16(Xs, Ximg, xi * 4);                   // group 1: X
  stage16(Es, E, n * lde * 4);                 // group 2: E (waited for after w)
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * LR_ROWS;
  for (int e = t; e < LR_ROWS * n; e += LR_NT) {
    const int r = e / n, k = e - r * n;
    const int64_t i = i0 + r;
    as[r][k] = i < I ? make_float2(Ah[i * lda + k], Al[i * lda + k]) : make_float2(0.f, 0.f);
  }
  stage_wait<1>();
  __syncthreads();
  // w for rows r0, r0 + 1 and columns j1 = u, j2 = n - 1 - u, over a quarter of k
  {
    const int ks = t >> 7, h = (t >> 6) & 1, u = t & 63;
    const int r0 = 2 * h;
    const int j1 = u, j2 = n - 1 - u;
    float s[2][2] = {}, c[2][2] = {};          // [row][column]
    if (j1 <= j2) {
      const int q = (j2 + LR_KS) / LR_KS;      // ceil((j2 + 1) / LR_KS)
      const int k0 = ks * q, k1 = min(k0 + q, j2 + 1);
#pragma unroll 2
      for (int k = k0; k < k1; ++k) {
        const float2 a0 = as[r0][k], a1 = as[r0 + 1][k];
        const float x2 = Xs[k * np + j2];
        dot2_add(s[0][1], c[0][1], x2, a0.x, a0.y);
        dot2_add(s[1][1], c[1][1], x2, a1.x, a1.y);
        if (k <= j1) {
          const float x1 = Xs[k * np + j1];
          dot2_add(s[0][0], c[0][0], x1, a0.x, a0.y);
          dot2_add(s[1][0], c[1][0], x1, a1.x, a1.y);
        }
      }
    }
    float* pp = part[ks][t & 127];
    pp[0] = s[0][0]; pp[1] = c[0][0]; pp[2] = s[0][1]; pp[3] = c[0][1];
    pp[4] = s[1][0]; pp[5] = c[1][0]; pp[6] = s[1][1]; pp[7] = c[1][1];
  }
  __syncthreads();
  // quarters added in order; w.w per row in double-float; w rounded to FP32 into wv
  float ws[4] = {};                             // (s, c) of rows r0, r0 + 1
  if (t < 128) {
    const int h = t >> 6, u = t & 63;
    const int r0 = 2 * h;
    const int j1 = u, j2 = n - 1 - u;
    if (j1 <= j2) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int col = 0; col < 2; ++col) {
          if (col == 0 && j1 == j2) continue;   // the middle column, counted once
          float ss = 0.f, sc = 0.f;
#pragma unroll
          for (int k = 0; k < LR_KS; ++k) {
            float tt, qq;
            two_sum(ss, part[k][t][4 * q + 2 * col], tt, qq);
            ss = tt;
            sc += part[k][t][4 * q + 2 * col + 1] + qq;
          }
          float hh, ll;
          renorm(ss, sc, hh, ll);
          dot2_add(ws[2 * q], ws[2 * q + 1], hh, hh, ll);
          ws[2 * q + 1] = fmaf(hh, ll, ws[2 * q + 1]);
          wv[r0 + q][col == 0 ? j1 : j2] = hh;
        }
      }
    }
    warp_sum2(ws[0], ws[1]);
    warp_sum2(ws[2], ws[3]);
    if (lane == 0)
#pragma unroll
      for (int m = 0; m < 4; ++m) red[warp][m] = ws[m];
  }
  stage_wait<0>();
  __syncthreads();
  // the double-float w.w of row t (t < LR_ROWS): warps 2h, 2h + 1 hold rows 2h, 2h + 1
  float wsr = 0.f, wcr = 0.f;
  if (t < LR_ROWS) {
    const int h = t >> 1, q = t & 1;
#pragma unroll
    for (int w2 = 0; w2 < 2; ++w2) {
      float tt, qq;
      two_sum(wsr, red[2 * h + w2][2 * q], tt, qq);
      wsr = tt;
      wcr += red[2 * h + w2][2 * q + 1] + qq;
    }
  }
  // v1 = E w, v2 = E v1, v3 = E v2; thread t: row r = t / 128, column j = t % 128
  const int r = t >> 7, j = t & 127;
  float d[6] = {};                             // d[k-1] = w_r^T E^k w_r (this column)
  float vprev = j < n ? wv[r][j] : 0.f;
  for (int m = 1; m <= 3; ++m) {
    if (m > nmv) break;
    float v = 0.f;
    if (j < n) {
      float va = 0.f, vb = 0.f, vc = 0.f, vd = 0.f;
      int k = 0;
      for (; k + 4 <= n; k += 4) {
        va = fmaf(Es[k * lde + j], wv[r][k], va);
        vb = fmaf(Es[(k + 1) * lde + j], wv[r][k + 1], vb);
        vc = fmaf(Es[(k + 2) * lde + j], wv[r][k + 2], vc);
        vd = fmaf(Es[(k + 3) * lde + j], wv[r][k + 3], vd);
      }
      for (; k < n; ++k) va = fmaf(Es[k * lde + j], wv[r][k], va);
      v = (va + vb) + (vc + vd);
    }
    __syncthreads();                           // every thread is done reading wv
    if (j < n) {
      if (m == 1) { d[0] = vprev * v; d[1] = v * v; }
      if (m == 2) { d[2] = vprev * v; d[3] = v * v; }
      if (m == 3) { d[4] = vprev * v; d[5] = v * v; }
      wv[r][j] = v;
      vprev = v;
    }
    __syncthreads();
  }
  // per-row sums of d: warps 4r .. 4r + 3 hold row r
#pragma unroll
  for (int k = 0; k < 6; ++k) d[k] = warp_sum(d[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) red[warp][k] = d[k];
  __syncthreads();
  if (t < LR_ROWS && i0 + t < I) {
    float tot[6] = {};
#pragma unroll
    for (int w4 = 0; w4 < 4; ++w4)
#pragma unroll
      for (int k = 0; k < 6; ++k) tot[k] += red[4 * t + w4][k];
    // alternating series, smallest terms first
    const float corr = tot[5] - tot[4] + tot[3] - tot[2] + tot[1] - tot[0];
    ell[i0 + t] = static_cast<double>(wsr) + (static_cast<double>(wcr) + static_cast<double>(corr));
  }
  // the CTA that finishes last forms p and the CDF
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    s_last = (atomicAdd(ep.counter, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (s_last) {
    __threadfence();
    cdf_epilogue_nw<LR_NT / 32>(ep, ell, I);
    if (threadIdx.x == 0) *ep.counter = 0u;
  }
}

size_t lev_rows_smem(int n) {
  return (static_cast<size_t>(pad4(n * (n + 1))) + static_cast<size_t>(n) * pad4(n)) * 4;
}

__global__ void k_planes_sum(const float* __restrict__ hi, const float* __restrict__ lo,
                             int64_t count, double* __restrict__ dst) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[e] = static_cast<double>(hi[e]) + static_cast<double>(lo[e]);
}

__global__ void k_copy_int(const int* src, int v, int* dst) { *dst = src ? *src : v; }

}  // namespace

cudaError_t launch_planes_sum(const float* hi, const float* lo, int64_t count, double* dst,
                              cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4 * sm_count()) blocks = 4 * sm_count();
  k_planes_sum<<<static_cast<unsigned>(blocks), 256, 0, st>>>(hi, lo, count, dst);
  return cudaGetLastError();
}

cudaError_t launch_copy_int(const int* src, int v, int* dst, cudaStream_t st) {
  k_copy_int<<<1, 1, 0, st>>>(src, v, dst);
  return cudaGetLastError();
}

int gram_dd_splits(int64_t I, int64_t* chunk) {
  int64_t c = (I + 7) / 8;                      // about 8 splits of at least 32 rows
  c = (c + GDK - 1) / GDK * GDK;
  *chunk = c;
  return static_cast<int>((I + c - 1) / c);
}

size_t gram_dd_partial_floats(int64_t I, int n) {
  int64_t chunk;
  const int nt = (n + GD - 1) / GD;
  return static_cast<size_t>(gram_dd_splits(I, &chunk)) * (nt * (nt + 1) / 2) * GD * GD;
}

cudaError_t launch_gram_dd(const float* Ah, const float* Al, int64_t I, int n, int64_t lda_a,
                           float* ph, float* pl, unsigned* cnt, float* kh, float* kl, int lda,
                           double* k64, cudaStream_t st) {
  int64_t chunk;
  const int splits = gram_dd_splits(I, &chunk);
  const int nt = (n + GD - 1) / GD;
  k_gram_dd<<<dim3(nt * (nt + 1) / 2, splits), GDNT, 0, st>>>(Ah, Al, I, n, lda_a, chunk, splits,
                                                              ph, pl, cnt, kh, kl, lda, k64);
  return cudaGetLastError();
}

bool lev_precond_fits(int64_t I, int n) { return n >= 4 && n <= kMaxPre && I >= n; }

int lev_precond_ctas(int n) {
  const int t = (n + LT - 1) / LT;
  return t * (t + 1) / 2;
}

cudaError_t launch_lev_precond(int stage, const LevPrecond& lp, int n, int64_t I,
                               const float* Ah, const float* Al, int64_t lda, double* ell,
                               const CdfEpilogue& ep, cudaStream_t st) {
  if (!lev_precond_fits(I, n) || lp.lda_k != pad4(n)) return cudaErrorInvalidValue;
  const int ld = pad4(n);
  const int nt = (n + LT - 1) / LT;
  switch (stage) {
    case 0: {
      const double eps32 = 1.1920928955078125e-07;
      k_chol_inv<<<1, chol_inv_threads(n), 0, st>>>(n, static_cast<float>(n * eps32), lp.K_hi,
                                                    lp.lda_k, lp.Ximg, lp.state);
      return cudaGetLastError();
    }
    case 1:
      k_lev_u<<<dim3(nt, nt), dim3(LT, LT), 0, st>>>(n, lp.K_hi, lp.K_lo, lp.lda_k, lp.Ximg,
                                                     lp.state, lp.Uh, lp.Ul, ld);
      return cudaGetLastError();
    case 2:
      k_lev_e<<<lev_precond_ctas(n), dim3(LT, LT), 0, st>>>(n, lp.Uh, lp.Ul, ld, lp.Ximg,
                                                           lp.state, lp.E, ld, lp.esq);
      return cudaGetLastError();
    case 3: {
      const unsigned rb = static_cast<unsigned>((I + LR_ROWS - 1) / LR_ROWS);
      k_lev_rows<<<rb, LR_NT, lev_rows_smem(n), st>>>(n, I, Ah, Al, lda, lp.Ximg, lp.E, ld,
                                                        lp.esq, lev_precond_ctas(n), lp.state,
                                                        ell, ep, lp.tau);
      return cudaGetLastError();
    }
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t lev_precond_attributes() {
  return cudaFuncSetAttribute(k_lev_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(lev_rows_smem(kMaxPre)));
}

}  // namespace trk
