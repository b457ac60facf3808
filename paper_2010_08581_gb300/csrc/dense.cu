// Dense TR-ALS (Alg. 1) on the same least-squares path as the sampled method: every row of
// G_[2]^{!=n} and of X_[n]^T, each with weight 1, instead of J sampled ones (Def. 5 with
// S = I). Rows are taken in the row-major order of the modes other than n (the last mode
// fastest), which is the memory order of X: row r = pre * P_post + post, where X is viewed as
// [P_pre][I_n][P_post].
#include "common.cuh"

namespace trk {
namespace {

// Row r -> its multi-index in ring order (position m holds mode (n + 1 + m) % N).
__global__ void __launch_bounds__(256) k_enumerate(int N, int n, DenseDims d, int64_t P,
                                                   int32_t* __restrict__ idx) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= P) return;
  int64_t rest = r;
  for (int mode = N - 1; mode >= 0; --mode) {
    if (mode == n) continue;
    const int64_t i = rest % d.I[mode];
    rest /= d.I[mode];
    const int m = (mode - n - 1 + N) % N;
    idx[r * (N - 1) + m] = static_cast<int32_t>(i);
  }
}

// Y[pre * P_post + q][i] = X[pre][i][q] (a batched transpose of the I_n x P_post slabs),
// through 32 x 32 shared-memory tiles: reads coalesced along q, writes along i.
template <typename TX, typename TY>
__global__ void __launch_bounds__(256) k_unfold(const TX* __restrict__ X, int64_t Ppre,
                                                int64_t In, int64_t Ppost, TY* __restrict__ Y) {
  __shared__ TY tile[32][33];
  const int64_t q0 = static_cast<int64_t>(blockIdx.x) * 32, i0 = static_cast<int64_t>(blockIdx.y) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 32 per pass
  for (int64_t pre = blockIdx.z; pre < Ppre; pre += gridDim.z) {
    const TX* src = X + pre * In * Ppost;
    TY* dst = Y + pre * Ppost * In;
    for (int r = ty; r < 32; r += 8) {
      const int64_t i = i0 + r, q = q0 + tx;
      if (i < In && q < Ppost) tile[r][tx] = static_cast<TY>(src[i * Ppost + q]);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int64_t q = q0 + r, i = i0 + tx;
      if (q < Ppost && i < In) dst[q * In + i] = tile[tx][r];
    }
    __syncthreads();
  }
}

// Y = X with a type change (the last mode: X is already [P][I_n]).
template <typename TX, typename TY>
__global__ void __launch_bounds__(256) k_convert(const TX* __restrict__ X, int64_t count,
                                                 TY* __restrict__ Y) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    Y[e] = static_cast<TY>(X[e]);
}

template <typename TX, typename TY>
cudaError_t unfold_t(const TX* X, int64_t Ppre, int64_t In, int64_t Ppost, TY* Y,
                     cudaStream_t st) {
  if (Ppost == 1) {
    const int64_t count = Ppre * In;
    const unsigned blocks = static_cast<unsigned>(count / 256 + 1 < sm_count() * 16 ? count / 256 + 1 : sm_count() * 16);
    k_convert<TX, TY><<<blocks, 256, 0, st>>>(X, count, Y);
    return cudaGetLastError();
  }
  dim3 grid(static_cast<unsigned>((Ppost + 31) / 32), static_cast<unsigned>((In + 31) / 32),
            static_cast<unsigned>(Ppre < 65535 ? Ppre : 65535));
  k_unfold<TX, TY><<<grid, 256, 0, st>>>(X, Ppre, In, Ppost, Y);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_enumerate(int N, int n, const DenseDims& d, int32_t* idx, cudaStream_t st) {
  int64_t P = 1;
  for (int m = 0; m < N; ++m)
    if (m != n) P *= d.I[m];
  if (P <= 0) return cudaSuccess;
  k_enumerate<<<static_cast<unsigned>((P + 255) / 256), 256, 0, st>>>(N, n, d, P, idx);
  return cudaGetLastError();
}

cudaError_t launch_unfold(const void* X, bool x_f64, int N, int n, const DenseDims& d, void* Y,
                          bool y_f64, cudaStream_t st) {
  int64_t Ppre = 1, Ppost = 1;
  for (int m = 0; m < n; ++m) Ppre *= d.I[m];
  for (int m = n + 1; m < N; ++m) Ppost *= d.I[m];
  const int64_t In = d.I[n];
  // grid.x, grid.y <= 65535 tiles: checked by the caller (dense_fits)
  if (x_f64 && y_f64)
    return unfold_t(static_cast<const double*>(X), Ppre, In, Ppost, static_cast<double*>(Y), st);
  if (x_f64)
    return unfold_t(static_cast<const double*>(X), Ppre, In, Ppost, static_cast<float*>(Y), st);
  if (y_f64)
    return unfold_t(static_cast<const float*>(X), Ppre, In, Ppost, static_cast<double*>(Y), st);
  return unfold_t(static_cast<const float*>(X), Ppre, In, Ppost, static_cast<float*>(Y), st);
}

}  // namespace trk
