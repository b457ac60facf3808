// Relative-error partial sums ||TR(cores) - X||_F^2 and ||X||_F^2 (Sec. 4.1, Sec. 5.1)
// without forming TR(cores), shared by the single-problem kernels and the served fit.
//
// The modes are split at s (1 <= s <= N-1): X is viewed as a rows x cols matrix with
// rows = prod_{m<s} I_m and cols = prod_{m>=s} I_m (row-major X). By eq. 1,
//   TR(p, q) = trace(P_left(p) P_right(q)),
//   P_left(p)  = G^(0)(:, i_0, :) ... G^(s-1)(:, i_{s-1}, :)    (R_{N-1} x R_{s-1}),
//   P_right(q) = G^(s)(:, i_s, :) ... G^(N-1)(:, i_{N-1}, :)    (R_{s-1} x R_{N-1}),
// so TR(p, q) = sum_e V_p[e] W_q[e] over e = b * R_{N-1} + a with V_p[e] = P_left[a][b] and
// W_q[e] = P_right[b][a]: one dense contraction with K = R_{N-1} R_{s-1} <= 256.
//
// W is formed once per evaluation (fit_right_warp, e-major: W^T[e][q]) and V per block of FL
// rows in shared memory. Each thread computes an MI x MJ register tile of TR from two
// vector loads per e; squares of (X - TR) and of X are summed per tile in X's precision and
// accumulated across tiles in FP64 per thread. The
// split is chosen so that cols is large enough to amortise the row chains while W^T stays
// small (fit_split).
#pragma once

#include "common.cuh"

namespace trk {

constexpr int FNT = 256;                       // threads of a fit CTA
constexpr int64_t kFitMinCols = 256;           // grow cols (move s left) up to this
constexpr int64_t kFitMaxRight = 1ll << 22;    // max elements of W^T (cols * K)

template <typename T>
struct FitTile;
template <>
struct FitTile<float> {    // 64 x 64 outputs per tile, 4 x 4 per thread
  static constexpr int FL = 64, FI = 64, MI = 4, MJ = 4;
};
template <>
struct FitTile<double> {   // 32 x 32 outputs per tile, 2 x 2 per thread
  static constexpr int FL = 32, FI = 32, MI = 2, MJ = 2;
};

struct FitSplit {
  int s;          // first mode of the right group
  int K;          // R_{N-1} * R_{s-1}
  int64_t rows, cols;
};

__host__ __device__ inline FitSplit fit_split(int N, const int64_t* dims, const int* ranks) {
  FitSplit f;
  f.s = N - 1;
  f.cols = dims[N - 1];
  while (f.s > 1 && f.cols < kFitMinCols) {
    const int64_t c2 = f.cols * dims[f.s - 1];
    const int64_t k2 = static_cast<int64_t>(ranks[N - 1]) * ranks[f.s - 2];
    if (c2 * k2 > kFitMaxRight) break;
    f.s -= 1;
    f.cols = c2;
  }
  f.rows = 1;
  for (int m = 0; m < f.s; ++m) f.rows *= dims[m];
  f.K = ranks[N - 1] * ranks[f.s - 1];
  return f;
}

// Dynamic shared memory of a fit CTA for contraction length K.
template <typename T>
__host__ __device__ constexpr size_t fit_smem_bytes(int K) {
  return static_cast<size_t>(K) * (FitTile<T>::FL + FitTile<T>::FI) * sizeof(T);
}

// Loads `n` consecutive elements (n = 2 or 4, 16-byte aligned) from shared memory.
template <typename T, int n>
__device__ __forceinline__ void load_vec(const T* p, T* out) {
  if constexpr (sizeof(T) == 4 && n == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else if constexpr (sizeof(T) == 8 && n == 2) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    out[0] = v.x; out[1] = v.y;
  } else {
#pragma unroll
    for (int u = 0; u < n; ++u) out[u] = p[u];
  }
}

// Product of the lateral slices of modes m0..m1-1 at indices ii[m] into S (row-major
// R_{m0-1} x R_{m1-1}), one warp; G is per-warp scratch. Returns the column count.
template <typename T>
__device__ __forceinline__ int warp_slice_product(const FitArgs& a, int m0, int m1,
                                                  const int64_t* ii, T* S, T* G, int lane) {
  const int N = a.N;
  int rows = a.ranks[(m0 - 1 + N) % N], cols = a.ranks[m0];
  {
    const double* src = a.core[m0] + ii[m0] * rows * cols;
    for (int e = lane; e < rows * cols; e += 32) S[e] = static_cast<T>(src[e]);
  }
  for (int m = m0 + 1; m < m1; ++m) {
    const int rr = a.ranks[m];
    const double* src = a.core[m] + ii[m] * cols * rr;
    for (int e = lane; e < cols * rr; e += 32) G[e] = static_cast<T>(src[e]);
    __syncwarp();
    T acc[kMaxL / 32];
#pragma unroll
    for (int q = 0; q < kMaxL / 32; ++q) {
      const int e = lane + 32 * q;
      T s = T(0);
      if (e < rows * rr) {
        const int r = e / rr, c = e - r * rr;
        for (int t = 0; t < cols; ++t) s += S[r * cols + t] * G[t * rr + c];
      }
      acc[q] = s;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kMaxL / 32; ++q) {
      const int e = lane + 32 * q;
      if (e < rows * rr) S[e] = acc[q];
    }
    __syncwarp();
    cols = rr;
  }
  return cols;
}

// W^T[e][q] = P_right(q)[b][a] (e = b * R_{N-1} + a: the row-major index of P_right) for
// column q, one warp; S and G are per-warp scratch of kMaxL elements.
template <typename T>
__device__ __forceinline__ void fit_right_warp(const FitArgs& a, const FitSplit& f, int64_t q,
                                               T* __restrict__ WT, T* S, T* G, int lane) {
  const int N = a.N;
  int64_t ii[kMaxModes];
  int64_t rem = q;
  for (int m = N - 1; m >= f.s; --m) { ii[m] = rem % a.dims[m]; rem /= a.dims[m]; }
  warp_slice_product<T>(a, f.s, N, ii, S, G, lane);
  __syncwarp();
  for (int e = lane; e < f.K; e += 32) WT[e * f.cols + q] = S[e];
  __syncwarp();
}

// V_p[e] (e = b * R_{N-1} + a, V_p[e] = P_left(p)[a][b]) for the rows p0 .. p0 + nb - 1 of a
// block and the entries e0 <= e < e1, handed to put(ll, e, value) (rows past the end give
// zeros). All threads of the CTA call it; it ends with a CTA barrier.
//
// Rows p = pre * J + last (J = I_{s-1}) share the prefix G^(0) .. G^(s-2) of their slice
// chain, and consecutive rows mostly share it: each distinct prefix of the block is formed
// once by one warp (into chain[w]), and every (row, b) item then finishes its column b of
// P_left = prefix * G^(s-1)(:, last, :) in registers. The products and their summation order
// are those of a per-row chain, so V is the same. Blocks with more than 8 prefixes (J < 16)
// form every row's chain with one warp.
template <typename T, typename Put>
__device__ void build_left(const FitArgs& a, const FitSplit& f, int64_t p0, int nb, int e0,
                           int e1, T (*chain)[kMaxL], T (*slice)[kMaxL], Put put) {
  const int N = a.N, s = f.s;
  const int K = e1 < f.K ? e1 : f.K;   // entries K .. e1 - 1 are the caller's padding
  const int Rlast = a.ranks[N - 1], Rs = a.ranks[s - 1];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t rows = f.rows;
  const int64_t pend = (p0 + nb < rows) ? p0 + nb : rows;
  if (s == 1) {   // P_left(p) is the slice G^(0)(:, p, :) itself
    const int w = K - e0;
    for (int it = tid; it < nb * w; it += FNT) {
      const int ll = it / w, e = e0 + (it - ll * w);
      const int64_t p = p0 + ll;
      const int b = e / Rlast, aa = e - b * Rlast;
      put(ll, e, p < rows ? static_cast<T>(a.core[0][(p * Rlast + aa) * Rs + b]) : T(0));
    }
    __syncthreads();
    return;
  }
  const int64_t J = a.dims[s - 1];
  const int64_t pre_lo = p0 / J;
  const int npre = pend > p0 ? static_cast<int>((pend - 1) / J - pre_lo + 1) : 0;
  if (npre > FNT / 32) {
    // many short prefixes: one warp per row forms the whole chain
    for (int ll = warp; ll < nb; ll += FNT / 32) {
      const int64_t p = p0 + ll;
      if (p >= rows) {
        for (int e = e0 + lane; e < K; e += 32) put(ll, e, T(0));
        continue;
      }
      int64_t ii[kMaxModes];
      int64_t rem = p;
      for (int m = s - 1; m >= 0; --m) { ii[m] = rem % a.dims[m]; rem /= a.dims[m]; }
      T* S = chain[warp];
      const int rs = warp_slice_product<T>(a, 0, s, ii, S, slice[warp], lane);
      __syncwarp();
      for (int e = e0 + lane; e < K; e += 32) {
        const int b = e / Rlast, aa = e - b * Rlast;
        put(ll, e, S[aa * rs + b]);
      }
      __syncwarp();
    }
    __syncthreads();
    return;
  }
  const int Rm = a.ranks[s - 2];   // the rank between the prefix and G^(s-1)
  if (warp < npre) {
    int64_t ii[kMaxModes];
    int64_t rem = pre_lo + warp;
    for (int m = s - 2; m >= 0; --m) { ii[m] = rem % a.dims[m]; rem /= a.dims[m]; }
    warp_slice_product<T>(a, 0, s - 1, ii, chain[warp], slice[warp], lane);   // Rlast x Rm
  }
  __syncthreads();
  const double* Gs = a.core[s - 1];
  // columns b whose entries b * Rlast .. b * Rlast + Rlast - 1 meet [e0, K)
  const int b0 = e0 / Rlast, b1 = (K + Rlast - 1) / Rlast;
  const int nbc = b1 - b0;
  for (int it = tid; it < nb * nbc; it += FNT) {
    const int ll = it / nbc, b = b0 + (it - ll * nbc);
    const int64_t p = p0 + ll;
    const int a0 = e0 > b * Rlast ? e0 - b * Rlast : 0;
    const int a1 = K < (b + 1) * Rlast ? K - b * Rlast : Rlast;
    if (p >= rows) {
      for (int aa = a0; aa < a1; ++aa) put(ll, b * Rlast + aa, T(0));
      continue;
    }
    const int64_t pre = p / J, last = p - pre * J;
    const T* P = chain[pre - pre_lo];
    const double* g = Gs + last * Rm * Rs + b;   // column b of G^(s-1)(:, last, :)
    T gc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) gc[c] = c < Rm ? static_cast<T>(g[c * Rs]) : T(0);
    for (int aa = a0; aa < a1; ++aa) {
      const T* pr = P + aa * Rm;
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < Rm) acc += pr[c] * gc[c];
      put(ll, b * Rlast + aa, acc);
    }
  }
  __syncthreads();
}

// Accumulates the squared residual (se) and ||X||^2 (sx) over the row blocks
// first, first + stride, ... All threads of the CTA must call it. `chain` and `slice` are
// per-warp scratch of kMaxL elements (8 warps); `dyn` holds fit_smem_bytes<T>(f.K).
template <typename T>
__device__ void fit_blocks(const FitArgs& a, const FitSplit& f, const T* __restrict__ X,
                           const T* __restrict__ WT, int64_t first, int64_t stride,
                           unsigned char* dyn, T (*chain)[kMaxL], T (*slice)[kMaxL],
                           double& se, double& sx) {
  constexpr int FL = FitTile<T>::FL, FI = FitTile<T>::FI;
  constexpr int MI = FitTile<T>::MI, MJ = FitTile<T>::MJ;
  constexpr int TX = FI / MJ;   // threads along the columns (16)
  static_assert((FL / MI) * (FI / MJ) == FNT, "one register tile per thread");
  static_assert(FL / MI == 16, "16 swizzled groups per row of V^T");
  // Row e of V^T stores its 16 groups of MI entries in the order g ^ (e & 15): the per-row
  // column writes of the chain phase spread over the banks, each group stays contiguous.
  auto vpos = [](int e, int ll) { return e * FL + (((ll / MI) ^ (e & 15)) * MI) + ll % MI; };
  const int N = a.N;
  const int K = f.K;
  T* Vt = reinterpret_cast<T*>(dyn);   // [K][FL]
  T* Qt = Vt + K * FL;                 // [K][FI]
  const int64_t rows = f.rows, cols = f.cols;
  const int ty = threadIdx.x / TX, tx = threadIdx.x % TX;
  const bool vec_ok = sizeof(T) == 4 && (cols % 4) == 0 &&
                      (reinterpret_cast<uintptr_t>(WT) % 16) == 0;

  for (int64_t blk = first; blk * FL < rows; blk += stride) {
    const int64_t p0 = blk * FL;
    // 1. V^T for the FL rows of the block.
    build_left<T>(a, f, p0, FL, 0, K, chain, slice,
                  [&](int ll, int e, T v) { Vt[vpos(e, ll)] = v; });
    // 2. TR(p, q) for tiles of FI columns, MI x MJ per thread.
    for (int64_t q0 = 0; q0 < cols; q0 += FI) {
      const int nq = static_cast<int>((cols - q0 < FI) ? cols - q0 : FI);
      if (vec_ok && nq == FI) {
        for (int o = threadIdx.x; o < K * (FI / 4); o += FNT) {
          const int e = o / (FI / 4), c4 = o - e * (FI / 4);
          *reinterpret_cast<float4*>(Qt + e * FI + 4 * c4) =
              *reinterpret_cast<const float4*>(WT + e * cols + q0 + 4 * c4);
        }
      } else {
        for (int o = threadIdx.x; o < K * FI; o += FNT) {
          const int e = o / FI, iq = o - e * FI;
          Qt[o] = iq < nq ? WT[e * cols + q0 + iq] : T(0);
        }
      }
      __syncthreads();
      T acc[MI][MJ];
#pragma unroll
      for (int u = 0; u < MI; ++u)
#pragma unroll
        for (int v = 0; v < MJ; ++v) acc[u][v] = T(0);
      const T* qp = Qt + tx * MJ;
#pragma unroll 4
      for (int e = 0; e < K; ++e) {
        T vv[MI], qq[MJ];
        load_vec<T, MI>(Vt + e * FL + (ty ^ (e & 15)) * MI, vv);
        load_vec<T, MJ>(qp + e * FI, qq);
#pragma unroll
        for (int u = 0; u < MI; ++u)
#pragma unroll
          for (int v = 0; v < MJ; ++v) acc[u][v] += vv[u] * qq[v];
      }
      // The tile's squares are summed in T and added to the FP64 totals once per tile
      // (GB300's FP64 pipe is about 1/64 of its FP32 rate).
      T se_t = T(0), sx_t = T(0);
#pragma unroll
      for (int u = 0; u < MI; ++u) {
        const int64_t p = p0 + ty * MI + u;
        if (p >= rows) continue;
        const T* xr = X + p * cols + q0;
#pragma unroll
        for (int v = 0; v < MJ; ++v) {
          const int iq = tx * MJ + v;
          if (iq >= nq) continue;
          const T x = xr[iq];
          const T d = x - acc[u][v];
          se_t += d * d;
          sx_t += x * x;
        }
      }
      se += static_cast<double>(se_t);
      sx += static_cast<double>(sx_t);
      __syncthreads();
    }
  }
}

// Block sum of (se, sx) to thread 0; `red` holds 2 * (FNT / 32) doubles.
__device__ __forceinline__ void fit_block_reduce(double& se, double& sx, double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  if (lane == 0) { red[warp] = se; red[FNT / 32 + warp] = sx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < FNT / 32; ++w) { a0 += red[w]; a1 += red[FNT / 32 + w]; }
    se = a0;
    sx = a1;
  }
}

}  // namespace trk
