// Row a5: normal-equation contractions of the sampled LS (Alg. 2, LS step):
//   M = A~^T A~ (L x L),  B = A~^T Y~ (L x I),
// computed together as C = A~^T [A~ | Y~] with the J rows split into chunks; each chunk
// writes its own partial C so that the reduction order downstream is fixed (results do
// not depend on scheduling).
//
// SIMT tiles: 64 x 64 outputs per CTA, 16 rows of J per shared-memory stage, 4 x 4 outputs
// per thread. T = float accumulates in FP32 within a chunk; T = double in FP64.
#include "common.cuh"

namespace trk {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T>
__global__ void __launch_bounds__(NT) k_normal_eq(const T* __restrict__ A,
                                                  const T* __restrict__ Y, int64_t J, int L,
                                                  int64_t I, int64_t chunk,
                                                  T* __restrict__ partial,
                                                  const int64_t* __restrict__ jdev) {
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int64_t ldc = L + I;
  const int r0 = blockIdx.y * BM;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * BN;
  const int64_t j0 = static_cast<int64_t>(blockIdx.z) * chunk;
  const int64_t Jr = jdev ? (*jdev < J ? *jdev : J) : J;
  const int64_t j1 = (j0 + chunk < Jr) ? j0 + chunk : Jr;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);

  for (int64_t jb = j0; jb < j1; jb += BK) {
    // 16 x 64 elements of each tile, 4 per thread.
#pragma unroll
    for (int q = 0; q < (BK * BM) / NT; ++q) {
      const int e = threadIdx.x + q * NT;
      const int kk = e / BM, col = e % BM;
      const int64_t j = jb + kk;
      const int r = r0 + col;
      As[kk][col] = (j < j1 && r < L) ? A[j * L + r] : T(0);
      const int64_t c = c0 + col;
      T b = T(0);
      if (j < j1) {
        if (c < L) b = A[j * L + c];
        else if (c < ldc) b = Y[j * I + (c - L)];
      }
      Bs[kk][col] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
  T* out = partial + static_cast<int64_t>(blockIdx.z) * L * ldc;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = r0 + ty + 16 * u;
    if (r >= L) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t c = c0 + tx + 16 * v;
      if (c < ldc) out[static_cast<int64_t>(r) * ldc + c] = acc[u][v];
    }
  }
}

void plan(int64_t J, int L, int64_t I, int* splits, int64_t* chunk) {
  const int64_t tiles = ((L + BM - 1) / BM) * ((L + I + BN - 1) / BN);
  int64_t s = (4 * sm_count() + tiles - 1) / tiles;
  const int64_t maxs = (J + 63) / 64;  // at least 64 rows per chunk
  if (s > maxs) s = maxs;
  if (s < 1) s = 1;
  int64_t c = (J + s - 1) / s;
  c = (c + BK - 1) / BK * BK;
  s = (J + c - 1) / c;
  *splits = static_cast<int>(s);
  *chunk = c;
}

}  // namespace

size_t normal_eq_workspace(int64_t J, int L, int64_t I, bool f64, int* splits) {
  int64_t chunk;
  plan(J, L, I, splits, &chunk);
  return static_cast<size_t>(*splits) * L * (L + I) * (f64 ? 8 : 4);
}

cudaError_t launch_normal_eq(const void* A, const void* Y, bool f64, int64_t J, int L,
                             int64_t I, void* partial, int splits, cudaStream_t st,
                             const int64_t* jdev) {
  int s;
  int64_t chunk;
  plan(J, L, I, &s, &chunk);
  if (s != splits) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned>((L + I + BN - 1) / BN), (L + BM - 1) / BM, s);
  if (f64)
    k_normal_eq<double><<<grid, NT, 0, st>>>(static_cast<const double*>(A),
                                             static_cast<const double*>(Y), J, L, I, chunk,
                                             static_cast<double*>(partial), jdev);
  else
    k_normal_eq<float><<<grid, NT, 0, st>>>(static_cast<const float*>(A),
                                            static_cast<const float*>(Y), J, L, I, chunk,
                                            static_cast<float*>(partial), jdev);
  return cudaGetLastError();
}

}  // namespace trk
