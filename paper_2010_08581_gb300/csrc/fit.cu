// Relative error ||TR(cores) - X||_F / ||X||_F (Sec. 4.1) without forming TR(cores).
// X is viewed as a (prod_{m<N-1} I_m) x I_{N-1} matrix. For a block of 32 leading
// multi-indices l the slice product P_l = G^(0)(:, i_0, :) ... G^(N-2)(:, i_{N-2}, :) is
// built in shared memory (eq. 1 without the last core); then for every i in the last mode
// TR(l, i) = trace(P_l G^(N-1)(:, i, :)) = sum_e V_l[e] Q_i[e] with Q_i the contiguous
// slice i of the last core and V_l[c*Rr + a] = P_l[a][c]. Squares of (X - TR) and of X are
// accumulated in FP64 per CTA.
#include "common.cuh"

namespace trk {
namespace {

constexpr int FL = 32;   // leading multi-indices per CTA
constexpr int FI = 32;   // last-mode indices per inner tile
constexpr int FNT = 256;

template <typename T>
__global__ void __launch_bounds__(FNT) k_fit(FitArgs a, const T* __restrict__ X, int64_t lead,
                                             double* __restrict__ partial, int blocks) {
  extern __shared__ __align__(16) unsigned char fit_smem_raw[];
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  __shared__ double red[2][FNT / 32];
  const int N = a.N;
  const int Rl_last = a.ranks[N - 2], Rr_last = a.ranks[N - 1];
  const int Lq = Rl_last * Rr_last;
  T* V = reinterpret_cast<T*>(fit_smem_raw);             // [FL][Lq]
  T* Qs = V + FL * Lq;                                    // [FI][Lq]
  const int64_t Ilast = a.dims[N - 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double se = 0.0, sx = 0.0;

  for (int64_t blk = blockIdx.x; blk * FL < lead; blk += gridDim.x) {
    const int64_t l0 = blk * FL;
    // 1. slice products for the FL leading indices, one warp per index.
    for (int ll = warp; ll < FL; ll += FNT / 32) {
      const int64_t l = l0 + ll;
      if (l >= lead) {
        for (int e = lane; e < Lq; e += 32) V[ll * Lq + e] = T(0);
        continue;
      }
      // decode l into (i_0..i_{N-2}), row-major (last leading mode fastest)
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
      // S is rows x cols = Rr_last x Rl_last (P[a][c]); V[c*Rr + a] = P[a][c].
      for (int e = lane; e < Lq; e += 32) {
        const int c = e / Rr_last, aa = e - c * Rr_last;
        V[ll * Lq + e] = S[aa * cols + c];
      }
      __syncwarp();
    }
    __syncthreads();
    // 2. TR(l, i) for tiles of the last mode.
    for (int64_t i0 = 0; i0 < Ilast; i0 += FI) {
      const int ni = static_cast<int>((Ilast - i0 < FI) ? Ilast - i0 : FI);
      for (int e = threadIdx.x; e < ni * Lq; e += FNT)
        Qs[e] = static_cast<T>(a.core[N - 1][(i0 * Lq) + e]);
      __syncthreads();
      for (int o = threadIdx.x; o < FL * FI; o += FNT) {
        const int ll = o / FI, iq = o - ll * FI;
        const int64_t l = l0 + ll;
        if (l >= lead || iq >= ni) continue;
        T s = T(0);
        const T* v = V + ll * Lq;
        const T* q = Qs + iq * Lq;
        for (int e = 0; e < Lq; ++e) s += v[e] * q[e];
        const double x = static_cast<double>(X[l * Ilast + i0 + iq]);
        const double d = x - static_cast<double>(s);
        se += d * d;
        sx += x * x;
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  if (lane == 0) { red[0][warp] = se; red[1][warp] = sx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < FNT / 32; ++w) { a0 += red[0][w]; a1 += red[1][w]; }
    partial[blockIdx.x] = a0;
    partial[blocks + blockIdx.x] = a1;
  }
}

}  // namespace

size_t fit_workspace(const FitArgs& a, int* blocks) {
  int64_t lead = 1;
  for (int m = 0; m < a.N - 1; ++m) lead *= a.dims[m];
  int64_t b = (lead + FL - 1) / FL;
  if (b > 152 * 8) b = 152 * 8;
  *blocks = static_cast<int>(b);
  return static_cast<size_t>(2 * b) * sizeof(double);
}

cudaError_t launch_fit(const FitArgs& a, const void* X, bool x_f64, double* partial, int blocks,
                       cudaStream_t st) {
  int64_t lead = 1;
  for (int m = 0; m < a.N - 1; ++m) lead *= a.dims[m];
  if (x_f64) {
    const size_t dyn = static_cast<size_t>(FL + FI) * a.ranks[a.N - 2] * a.ranks[a.N - 1] * sizeof(double);
    k_fit<double><<<blocks, FNT, dyn, st>>>(a, static_cast<const double*>(X), lead, partial,
                                            blocks);
  } else {
    const size_t dyn = static_cast<size_t>(FL + FI) * a.ranks[a.N - 2] * a.ranks[a.N - 1] * sizeof(float);
    k_fit<float><<<blocks, FNT, dyn, st>>>(a, static_cast<const float*>(X), lead, partial,
                                           blocks);
  }
  return cudaGetLastError();
}

// The largest dynamic request of k_fit is (FL + FI) * kMaxL elements.
cudaError_t fit_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fit<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (FL + FI) * kMaxL * static_cast<int>(sizeof(double)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fit<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (FL + FI) * kMaxL * static_cast<int>(sizeof(float)));
}

cudaError_t cholesky_attributes();
cudaError_t trsm_attributes();
cudaError_t normal_eq_tc_attributes();
cudaError_t sample_chain_attributes();
cudaError_t batched_attributes();

cudaError_t init_kernel_attributes(const char** which) {
  cudaError_t e = cholesky_attributes();
  if (e != cudaSuccess) { *which = "cholesky"; return e; }
  e = trsm_attributes();
  if (e != cudaSuccess) { *which = "trsm"; return e; }
  e = normal_eq_tc_attributes();
  if (e != cudaSuccess) { *which = "normal_eq_tc"; return e; }
  e = sample_chain_attributes();
  if (e != cudaSuccess) { *which = "sample_chain"; return e; }
  e = batched_attributes();
  if (e != cudaSuccess) { *which = "batched"; return e; }
  e = fit_attributes();
  if (e != cudaSuccess) *which = "fit";
  return e;
}

}  // namespace trk
