// Relative-error partial sums ||TR(cores) - X||_F^2 and ||X||_F^2 (Sec. 5.1) without forming
// TR(cores), shared by the single-problem kernel and the served fit evaluation.
//
// X is viewed as a (prod_{m<N-1} I_m) x I_{N-1} matrix. For a block of FL leading
// multi-indices l the slice product P_l = G^(0)(:, i_0, :) ... G^(N-2)(:, i_{N-2}, :) is built
// in shared memory (eq. 1 without the last core); then for every i of the last mode
// TR(l, i) = trace(P_l G^(N-1)(:, i, :)) = sum_e V_l[e] Q_i[e], with Q_i the contiguous slice
// i of the last core and V_l[c * Rr + a] = P_l[a][c]. Both operands are staged e-major
// (V^T: Lq x FL, Q^T: Lq x FI) so that each thread computes an MI x MJ register tile of
// TR(l, i) from two vector loads per e. Row e of V^T stores its 16 groups of MI entries in
// the order g ^ (e & 15), which spreads the per-index column writes over the banks while
// keeping each group contiguous. Squares are accumulated in FP64 per thread.
#pragma once

#include "common.cuh"

namespace trk {

constexpr int FNT = 256;   // threads of a fit CTA

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

// Dynamic shared memory of a fit CTA for last-core slices of Lq = R_{N-2} R_{N-1} entries.
template <typename T>
__host__ __device__ constexpr size_t fit_smem_bytes(int Lq) {
  return static_cast<size_t>(Lq) * (FitTile<T>::FL + FitTile<T>::FI) * sizeof(T);
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

// Accumulates the squared residual (se) and ||X||^2 (sx) over the leading blocks
// first, first + stride, ... of X. All threads of the CTA must call it. `chain` and `slice`
// are per-warp scratch of kMaxL elements (8 warps); `dyn` holds fit_smem_bytes<T>(Lq).
template <typename T>
__device__ void fit_blocks(const FitArgs& a, const T* __restrict__ X, int64_t lead,
                           int64_t first, int64_t stride, unsigned char* dyn,
                           T (*chain)[kMaxL], T (*slice)[kMaxL], double& se, double& sx) {
  constexpr int FL = FitTile<T>::FL, FI = FitTile<T>::FI;
  constexpr int MI = FitTile<T>::MI, MJ = FitTile<T>::MJ;
  constexpr int TX = FI / MJ;   // threads along the last mode (16)
  static_assert((FL / MI) * (FI / MJ) == FNT, "one register tile per thread");
  static_assert(FL / MI == 16, "16 swizzled groups per row of V^T");
  auto vpos = [](int e, int ll) { return e * FL + (((ll / MI) ^ (e & 15)) * MI) + ll % MI; };
  const int N = a.N;
  const int Rl_last = a.ranks[N - 2], Rr_last = a.ranks[N - 1];
  const int Lq = Rl_last * Rr_last;
  T* Vt = reinterpret_cast<T*>(dyn);   // [Lq][FL]
  T* Qt = Vt + Lq * FL;                // [Lq][FI]
  const int64_t Ilast = a.dims[N - 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ty = threadIdx.x / TX, tx = threadIdx.x % TX;

  for (int64_t blk = first; blk * FL < lead; blk += stride) {
    const int64_t l0 = blk * FL;
    // 1. slice products of the FL leading indices, one warp per index.
    for (int ll = warp; ll < FL; ll += FNT / 32) {
      const int64_t l = l0 + ll;
      if (l >= lead) {
        for (int e = lane; e < Lq; e += 32) Vt[vpos(e, ll)] = T(0);
        continue;
      }
      int64_t rem = l;
      int64_t ii[kMaxModes];
      for (int m = N - 2; m >= 0; --m) { ii[m] = rem % a.dims[m]; rem /= a.dims[m]; }
      T* S = chain[warp];
      T* G = slice[warp];
      {
        const int rl = a.ranks[N - 1], rr = a.ranks[0];
        const double* src = a.core[0] + ii[0] * rl * rr;
        for (int e = lane; e < rl * rr; e += 32) S[e] = static_cast<T>(src[e]);
      }
      int rows = a.ranks[N - 1], cols = a.ranks[0];
      for (int m = 1; m <= N - 2; ++m) {
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
      // S is Rr_last x Rl_last (P[a][c]); V[c * Rr_last + a] = P[a][c].
      for (int e = lane; e < Lq; e += 32) {
        const int c = e / Rr_last, aa = e - c * Rr_last;
        Vt[vpos(e, ll)] = S[aa * cols + c];
      }
      __syncwarp();
    }
    __syncthreads();
    // 2. TR(l, i) for tiles of the last mode, MI x MJ per thread.
    const double* Qg = a.core[N - 1];
    for (int64_t i0 = 0; i0 < Ilast; i0 += FI) {
      const int ni = static_cast<int>((Ilast - i0 < FI) ? Ilast - i0 : FI);
      for (int o = threadIdx.x; o < FI * Lq; o += FNT) {
        const int e = o / FI, iq = o - e * FI;
        Qt[o] = iq < ni ? static_cast<T>(Qg[(i0 + iq) * Lq + e]) : T(0);
      }
      __syncthreads();
      T acc[MI][MJ];
#pragma unroll
      for (int u = 0; u < MI; ++u)
#pragma unroll
        for (int v = 0; v < MJ; ++v) acc[u][v] = T(0);
      const T* qp = Qt + tx * MJ;
#pragma unroll 4
      for (int e = 0; e < Lq; ++e) {
        T vv[MI], qq[MJ];
        load_vec<T, MI>(Vt + e * FL + (ty ^ (e & 15)) * MI, vv);
        load_vec<T, MJ>(qp + e * FI, qq);
#pragma unroll
        for (int u = 0; u < MI; ++u)
#pragma unroll
          for (int v = 0; v < MJ; ++v) acc[u][v] += vv[u] * qq[v];
      }
#pragma unroll
      for (int u = 0; u < MI; ++u) {
        const int64_t l = l0 + ty * MI + u;
        if (l >= lead) continue;
        const T* xr = X + l * Ilast + i0;
#pragma unroll
        for (int v = 0; v < MJ; ++v) {
          const int iq = tx * MJ + v;
          if (iq >= ni) continue;
          const double x = static_cast<double>(xr[iq]);
          const double d = x - static_cast<double>(acc[u][v]);
          se += d * d;
          sx += x * x;
        }
      }
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
