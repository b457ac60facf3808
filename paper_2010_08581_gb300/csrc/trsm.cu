// Triangular solves with a Cholesky factor L (n <= 256) for many vectors:
//   mode 0 (leverage rows, row a1): ell_v = || L^-1 a_v ||^2 -- row norms of Q = A R^-1 of
//           the Cholesky-based thin QR (Def. 3.3);
//   mode 1 (LS solve, row a6):      z_v = L^-T L^-1 b_v, written into the new core;
//   mode 2 (LS solve + one refinement step, row a6):
//           z = L^-T L^-1 b;  r = b - M z;  z += L^-T L^-1 r.
// One warp owns NB vectors; lane l holds rows l, l+32, ... of each in registers, so a
// substitution step is one shuffle broadcast plus independent FMAs. The factor (and M) are
// staged in shared memory in the compute type T with a padded row stride when they fit.
#include "common.cuh"

namespace trk {
namespace {

constexpr int QMAX = kMaxL / 32;  // 8 register rows per lane
constexpr int TW = 4;             // warps per CTA

template <typename T>
struct Factor {
  const T* s;            // shared: s[c*(n+1) + r] = L[r][c]   (may be null)
  const double* Lcol;    // global: Lcol[c*n + r] = L[r][c]
  const double* Lrow;    // global: Lrow[c*n + r] = L[c][r]
  int n;
  __device__ __forceinline__ T col(int c, int r) const {   // L[r][c]
    return s ? s[c * (n + 1) + r] : static_cast<T>(Lcol[c * n + r]);
  }
  __device__ __forceinline__ T row(int c, int r) const {   // L[c][r]
    return s ? s[r * (n + 1) + c] : static_cast<T>(Lrow[c * n + r]);
  }
};

template <typename T, int NB>
__device__ __forceinline__ T pick(const T (&x)[QMAX][NB], int q, int v) {
  T s = x[0][v];
#pragma unroll
  for (int u = 1; u < QMAX; ++u) s = (u == q) ? x[u][v] : s;
  return s;
}

template <typename T, int NB>
__device__ __forceinline__ void put(T (&x)[QMAX][NB], int q, int v, T val) {
#pragma unroll
  for (int u = 0; u < QMAX; ++u)
    if (u == q) x[u][v] = val;
}

// x <- L^-1 x
template <typename T, int NB>
__device__ __forceinline__ void forward(T (&x)[QMAX][NB], const Factor<T>& F, const T* inv,
                                        int lane) {
  const int n = F.n;
  for (int c = 0; c < n; ++c) {
    const int qc = c >> 5, lc = c & 31;
    const T ic = inv[c];
    T xc[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) {
      xc[v] = __shfl_sync(0xffffffffu, pick(x, qc, v), lc) * ic;
      if (lane == lc) put(x, qc, v, xc[v]);
    }
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int r = lane + 32 * q;
      if (q >= qc && r > c && r < n) {
        const T l = F.col(c, r);
#pragma unroll
        for (int v = 0; v < NB; ++v) x[q][v] -= l * xc[v];
      }
    }
  }
}

// x <- L^-T x
template <typename T, int NB>
__device__ __forceinline__ void backward(T (&x)[QMAX][NB], const Factor<T>& F, const T* inv,
                                         int lane) {
  const int n = F.n;
  for (int c = n - 1; c >= 0; --c) {
    const int qc = c >> 5, lc = c & 31;
    const T ic = inv[c];
    T zc[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) {
      zc[v] = __shfl_sync(0xffffffffu, pick(x, qc, v), lc) * ic;
      if (lane == lc) put(x, qc, v, zc[v]);
    }
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int r = lane + 32 * q;
      if (q <= qc && r < c) {
        const T l = F.row(c, r);
#pragma unroll
        for (int v = 0; v < NB; ++v) x[q][v] -= l * zc[v];
      }
    }
  }
}

template <typename T, int NB>
__global__ void __launch_bounds__(TW * 32) k_trsm(int n, const double* __restrict__ Lrow,
                                                  const double* __restrict__ Lcol,
                                                  const double* __restrict__ invdiag,
                                                  const int* __restrict__ info, int64_t nvec,
                                                  const double* __restrict__ rhs, int64_t ld,
                                                  int mode, const double* __restrict__ M,
                                                  int Rl, int Rr, double* __restrict__ core_out,
                                                  double* __restrict__ ell, int use_smem) {
  extern __shared__ __align__(16) unsigned char trsm_smem[];
  if (info && *info) return;
  T* inv = reinterpret_cast<T*>(trsm_smem);                       // n (padded to kMaxL)
  T* Ls = inv + kMaxL;                                            // n*(n+1) if staged
  T* Ms = Ls + (use_smem ? n * (n + 1) : 0);                      // n*(n+1) if staged, mode 2
  for (int c = threadIdx.x; c < n; c += blockDim.x) inv[c] = static_cast<T>(invdiag[c]);
  if (use_smem) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int c = e / n, r = e - (e / n) * n;
      Ls[c * (n + 1) + r] = static_cast<T>(Lcol[e]);
      if (mode == 2) Ms[c * (n + 1) + r] = static_cast<T>(M[e]);
    }
  }
  __syncthreads();
  Factor<T> F{use_smem ? Ls : nullptr, Lcol, Lrow, n};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t v0 = (static_cast<int64_t>(blockIdx.x) * TW + warp) * NB;
  if (v0 >= nvec) return;
  T x[QMAX][NB];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    const int r = lane + 32 * q;
#pragma unroll
    for (int v = 0; v < NB; ++v)
      x[q][v] = (r < n && v0 + v < nvec) ? static_cast<T>(rhs[(v0 + v) * ld + r]) : T(0);
  }
  forward(x, F, inv, lane);
  if (mode == 0) {
#pragma unroll
    for (int v = 0; v < NB; ++v) {
      T s = T(0);
#pragma unroll
      for (int q = 0; q < QMAX; ++q) s += x[q][v] * x[q][v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && v0 + v < nvec) ell[v0 + v] = static_cast<double>(s);
    }
    return;
  }
  backward(x, F, inv, lane);
  if (mode == 2) {
    // residual r = b - M z (M symmetric: column t of M = row t)
    T res[QMAX][NB];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int r = lane + 32 * q;
#pragma unroll
      for (int v = 0; v < NB; ++v)
        res[q][v] = (r < n && v0 + v < nvec) ? static_cast<T>(rhs[(v0 + v) * ld + r]) : T(0);
    }
    for (int t = 0; t < n; ++t) {
      const int qt = t >> 5, lt = t & 31;
      T zt[NB];
#pragma unroll
      for (int v = 0; v < NB; ++v) zt[v] = __shfl_sync(0xffffffffu, pick(x, qt, v), lt);
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int r = lane + 32 * q;
        if (r < n) {
          const T m = use_smem ? Ms[t * (n + 1) + r] : static_cast<T>(M[t * n + r]);
#pragma unroll
          for (int v = 0; v < NB; ++v) res[q][v] -= m * zt[v];
        }
      }
    }
    forward(res, F, inv, lane);
    backward(res, F, inv, lane);
#pragma unroll
    for (int q = 0; q < QMAX; ++q)
#pragma unroll
      for (int v = 0; v < NB; ++v) x[q][v] += res[q][v];
  }
  // new core: core[i][a][b] = z[a + Rl*b]
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    const int r = lane + 32 * q;
    if (r >= n) continue;
    const int a = r % Rl, b = r / Rl;
#pragma unroll
    for (int v = 0; v < NB; ++v)
      if (v0 + v < nvec) core_out[(v0 + v) * n + a * Rr + b] = static_cast<double>(x[q][v]);
  }
}

template <typename T, int NB>
cudaError_t run(int n, const double* Lrow, const double* Lcol, const double* invdiag,
                const int* info, int64_t nvec, const double* rhs, int64_t ld, int mode,
                const double* M, int Rl, int Rr, double* core_out, double* ell, cudaStream_t st) {
  const size_t mats = (mode == 2) ? 2 : 1;
  const size_t staged = (kMaxL + mats * n * (n + 1)) * sizeof(T);
  const int use_smem = staged <= 200 * 1024 ? 1 : 0;
  const size_t dyn = use_smem ? staged : kMaxL * sizeof(T);
  const int64_t per_cta = static_cast<int64_t>(TW) * NB;
  const int64_t blocks = (nvec + per_cta - 1) / per_cta;
  k_trsm<T, NB><<<static_cast<unsigned>(blocks), TW * 32, dyn, st>>>(
      n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Rl, Rr, core_out, ell, use_smem);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trsm(int mode, bool f32, int n, const double* Lrow, const double* Lcol,
                        const double* invdiag, const int* info, int64_t nvec, const double* rhs,
                        int64_t ld, const double* M, int Rl, int Rr, double* core_out,
                        double* ell, cudaStream_t st) {
  if (nvec <= 0) return cudaSuccess;
  if (f32)
    return run<float, 2>(n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Rl, Rr,
                         core_out, ell, st);
  return run<double, 1>(n, Lrow, Lcol, invdiag, info, nvec, rhs, ld, mode, M, Rl, Rr, core_out,
                        ell, st);
}

cudaError_t trsm_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_trsm<float, 2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_trsm<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024);
}

}  // namespace trk
