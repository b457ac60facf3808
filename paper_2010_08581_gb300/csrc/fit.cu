// Relative error ||TR(cores) - X||_F / ||X||_F (Sec. 5.1) of one problem: partial sums of
// the squared residual and of ||X||^2 per CTA (fit_body.cuh), reduced in a fixed order.
#include "fit_body.cuh"

namespace trk {
namespace {

template <typename T>
__global__ void __launch_bounds__(FNT) k_fit(FitArgs a, const T* __restrict__ X, int64_t lead,
                                             double* __restrict__ partial, int blocks) {
  extern __shared__ __align__(16) unsigned char fit_smem_raw[];
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  __shared__ double red[2 * (FNT / 32)];
  double se = 0.0, sx = 0.0;
  fit_blocks<T>(a, X, lead, blockIdx.x, gridDim.x, fit_smem_raw, chain, slice, se, sx);
  fit_block_reduce(se, sx, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = se;
    partial[blocks + blockIdx.x] = sx;
  }
}

int64_t lead_of(const FitArgs& a) {
  int64_t lead = 1;
  for (int m = 0; m < a.N - 1; ++m) lead *= a.dims[m];
  return lead;
}

}  // namespace

size_t fit_workspace(const FitArgs& a, int* blocks) {
  // FP32 tiles have 64 leading indices (FP64: 32); the grid is sized for the FP32 tiles.
  int64_t b = (lead_of(a) + FitTile<float>::FL - 1) / FitTile<float>::FL;
  if (b > 152 * 4) b = 152 * 4;
  if (b < 1) b = 1;
  *blocks = static_cast<int>(b);
  return static_cast<size_t>(2 * b) * sizeof(double);
}

cudaError_t launch_fit(const FitArgs& a, const void* X, bool x_f64, double* partial, int blocks,
                       cudaStream_t st) {
  const int64_t lead = lead_of(a);
  const int Lq = a.ranks[a.N - 2] * a.ranks[a.N - 1];
  if (x_f64)
    k_fit<double><<<blocks, FNT, fit_smem_bytes<double>(Lq), st>>>(
        a, static_cast<const double*>(X), lead, partial, blocks);
  else
    k_fit<float><<<blocks, FNT, fit_smem_bytes<float>(Lq), st>>>(
        a, static_cast<const float*>(X), lead, partial, blocks);
  return cudaGetLastError();
}

cudaError_t fit_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fit<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(fit_smem_bytes<double>(kMaxL)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fit<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(fit_smem_bytes<float>(kMaxL)));
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
