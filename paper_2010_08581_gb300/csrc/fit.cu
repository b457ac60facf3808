// Relative error ||TR(cores) - X||_F / ||X||_F (Sec. 5.1) of one problem: the right factors
// W^T of the mode split (fit_body.cuh), then partial sums of the squared residual and of
// ||X||^2 per CTA, reduced on the host in a fixed order.
#include "fit_tc.cuh"

namespace trk {
namespace {

template <typename T>
__global__ void __launch_bounds__(FNT) k_fit_right(FitArgs a, FitSplit f, T* __restrict__ WT) {
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = static_cast<int64_t>(blockIdx.x) * (FNT / 32) + warp;
  if (q >= f.cols) return;
  fit_right_warp<T>(a, f, q, WT, chain[warp], slice[warp], lane);
}

template <typename T>
__global__ void __launch_bounds__(FNT) k_fit(FitArgs a, FitSplit f, const T* __restrict__ X,
                                             const T* __restrict__ WT,
                                             double* __restrict__ partial, int blocks) {
  extern __shared__ __align__(16) unsigned char fit_smem_raw[];
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  __shared__ double red[2 * (FNT / 32)];
  double se = 0.0, sx = 0.0;
  fit_blocks<T>(a, f, X, WT, blockIdx.x, gridDim.x, fit_smem_raw, chain, slice, se, sx);
  fit_block_reduce(se, sx, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = se;
    partial[blocks + blockIdx.x] = sx;
  }
}

__global__ void __launch_bounds__(FNT) k_fit_right_tc(FitArgs a, FitSplit f,
                                                     unsigned char* __restrict__ WS) {
  __shared__ float chain[8][kMaxL];
  __shared__ float slice[8][kMaxL];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ncol = (f.cols + FTN - 1) / FTN * FTN;
  const int64_t q = static_cast<int64_t>(blockIdx.x) * (FNT / 32) + warp;
  if (q >= ncol) return;
  fit_right_tc_warp(a, f, q, WS, chain[warp], slice[warp], lane);
}

__global__ void __launch_bounds__(FNT, 1) k_fit_tc(FitArgs a, FitSplit f,
                                                   const float* __restrict__ X,
                                                   const unsigned char* __restrict__ WS,
                                                   double* __restrict__ partial, int blocks,
                                                   unsigned* err) {
  extern __shared__ __align__(1024) unsigned char fit_tc_raw[];
  __shared__ float chain[8][kMaxL];
  __shared__ float slice[8][kMaxL];
  __shared__ double red[2 * (FNT / 32)];
  __shared__ FitTcShared sh;
  double se = 0.0, sx = 0.0;
  fit_tc_blocks(a, f, X, WS, blockIdx.x, gridDim.x, fit_tc_raw, chain, slice, sh, err, se, sx);
  fit_block_reduce(se, sx, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = se;
    partial[blocks + blockIdx.x] = sx;
  }
}

FitSplit split_of(const FitArgs& a) { return fit_split(a.N, a.dims, a.ranks); }

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

size_t fit_workspace(const FitArgs& a, bool x_f64, int* blocks) {
  const FitSplit f = split_of(a);
  int64_t b = fit_row_blocks(f, x_f64);
  const int64_t cap = fit_use_tc(f, x_f64) ? sm_count() : sm_count() * 4;   // the tensor-core form: 1 CTA/SM
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  *blocks = static_cast<int>(b);
  const size_t es = x_f64 ? 8 : 4;
  const size_t right = fit_use_tc(f, x_f64) ? fit_tc_right_bytes(f)
                                            : static_cast<size_t>(f.cols) * f.K * es;
  return round256(static_cast<size_t>(2 * b) * sizeof(double)) + right;
}

cudaError_t launch_fit(const FitArgs& a, const void* X, bool x_f64, void* ws, int blocks,
                       unsigned* err, cudaStream_t st) {
  const FitSplit f = split_of(a);
  double* partial = static_cast<double*>(ws);
  char* wt = static_cast<char*>(ws) + round256(static_cast<size_t>(2 * blocks) * sizeof(double));
  const unsigned rb = static_cast<unsigned>((f.cols + FNT / 32 - 1) / (FNT / 32));
  if (x_f64) {
    double* WT = reinterpret_cast<double*>(wt);
    k_fit_right<double><<<rb, FNT, 0, st>>>(a, f, WT);
    k_fit<double><<<blocks, FNT, fit_smem_bytes<double>(f.K), st>>>(
        a, f, static_cast<const double*>(X), WT, partial, blocks);
  } else {
    if (fit_use_tc(f, false)) {
      unsigned char* WS = reinterpret_cast<unsigned char*>(wt);
      const int64_t ncol = (f.cols + FTN - 1) / FTN * FTN;
      k_fit_right_tc<<<static_cast<unsigned>((ncol + FNT / 32 - 1) / (FNT / 32)), FNT, 0, st>>>(
          a, f, WS);
      k_fit_tc<<<blocks, FNT, kFitTcSmem, st>>>(a, f, static_cast<const float*>(X), WS, partial,
                                                 blocks, err);
    } else {
      float* WT = reinterpret_cast<float*>(wt);
      k_fit_right<float><<<rb, FNT, 0, st>>>(a, f, WT);
      k_fit<float><<<blocks, FNT, fit_smem_bytes<float>(f.K), st>>>(
          a, f, static_cast<const float*>(X), WT, partial, blocks);
    }
  }
  return cudaGetLastError();
}

cudaError_t fit_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fit<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(fit_smem_bytes<double>(kMaxL)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fit_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kFitTcSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fit<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(fit_smem_bytes<float>(kMaxL)));
}

cudaError_t cholesky_attributes();
cudaError_t trsm_attributes();
cudaError_t normal_eq_tc_attributes();
cudaError_t sample_chain_attributes();
cudaError_t batched_attributes();
cudaError_t jacobi_attributes();
cudaError_t solve_inv_attributes();
cudaError_t merge_attributes();
cudaError_t lev_precond_attributes();

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
  e = jacobi_attributes();
  if (e != cudaSuccess) { *which = "jacobi"; return e; }
  e = solve_inv_attributes();
  if (e != cudaSuccess) { *which = "solve_inv"; return e; }
  e = merge_attributes();
  if (e != cudaSuccess) { *which = "merge"; return e; }
  e = lev_precond_attributes();
  if (e != cudaSuccess) { *which = "lev_precond"; return e; }
  e = fit_attributes();
  if (e != cudaSuccess) *which = "fit";
  return e;
}

}  // namespace trk
