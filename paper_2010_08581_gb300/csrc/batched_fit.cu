// Serving: the exact relative fit of every slot that completed a sweep (Sec. 5.1) and the
// stop rule of Sec. 4.1, for the batched slot table.
#include "batched_kern.cuh"
#include "fit_tc.cuh"

namespace trk {
namespace {

// ------------------------------------------------------------------------------------
// Serving: relative fit 1 - ||TR - X|| / ||X|| (Sec. 5.1) of every slot that completed a
// sweep in this tick, as kFitParts (or fewer) partial sums in a fixed order, then the stop
// rule (|fit_s - fit_{s-1}| < tol after two or more sweeps, or the sweep cap) and the step
// counters.
// ------------------------------------------------------------------------------------
// The slot's step is the last update of a sweep.
__device__ __forceinline__ bool fit_due(const BInst& d) {
  if (!d.slot) return false;
  const SlotState& s = *d.slot;
  return s.status == kSlotRunning && s.step >= 0 && s.step % d.N == d.N - 1;
}

// Partial sums of one slot's fit: one per CTA, at most kFitParts.
__device__ __forceinline__ int fit_parts(const FitSplit& f, bool xf64) {
  const int64_t nblk = fit_row_blocks(f, xf64);
  return nblk < kFitParts ? static_cast<int>(nblk) : kFitParts;
}

__device__ __forceinline__ void fit_args(const BInst& d, FitArgs& fa) {
  fa.N = d.N;
  for (int m = 0; m < d.N; ++m) {
    fa.core[m] = d.cores[m];
    fa.dims[m] = d.dims[m];
    fa.ranks[m] = d.ranks[m];
  }
}

constexpr int kFitRightCtas = 64;   // CTAs per slot forming the right factors

// Right factors of the fit: e-major W^T for the SIMT contraction, or the swizzled hi/lo
// tiles of the tensor-core contraction.
template <typename T>
__global__ void __launch_bounds__(FNT) kb_fit_right(const BInst* __restrict__ tab) {
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  __shared__ FitArgs fa;
  const BInst& d = tab[blockIdx.x];
  if (!fit_due(d)) return;
  if (threadIdx.x == 0) fit_args(d, fa);
  __syncthreads();
  const FitSplit f = fit_split(fa.N, fa.dims, fa.ranks);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t step = static_cast<int64_t>(gridDim.y) * (FNT / 32);
  const int64_t q0 = static_cast<int64_t>(blockIdx.y) * (FNT / 32) + warp;
  if constexpr (sizeof(T) == 4) {
    if (fit_use_tc(f, false)) {
      unsigned char* WS = static_cast<unsigned char*>(d.fitw);
      const int64_t ncol = (f.cols + FTN - 1) / FTN * FTN;
      for (int64_t q = q0; q < ncol; q += step)
        fit_right_tc_warp(fa, f, q, WS, chain[warp], slice[warp], lane);
      return;
    }
  }
  T* WT = static_cast<T*>(d.fitw);
  for (int64_t q = q0; q < f.cols; q += step)
    fit_right_warp<T>(fa, f, q, WT, chain[warp], slice[warp], lane);
}

// Slots whose contraction length K lies in (k_lo, k_hi] (two launches with different
// shared-memory sizes keep the common small-K case at several CTAs per SM).
template <typename T>
__global__ void __launch_bounds__(FNT) kb_fit(const BInst* __restrict__ tab, int k_lo, int k_hi) {
  extern __shared__ __align__(16) unsigned char fit_dyn[];
  __shared__ T chain[8][kMaxL];
  __shared__ T slice[8][kMaxL];
  __shared__ double red[2 * (FNT / 32)];
  __shared__ FitArgs fa;
  const BInst& d = tab[blockIdx.x];
  if (!fit_due(d)) return;
  if (threadIdx.x == 0) fit_args(d, fa);
  __syncthreads();
  const FitSplit f = fit_split(fa.N, fa.dims, fa.ranks);
  if (fit_use_tc(f, sizeof(T) == 8) || f.K <= k_lo || f.K > k_hi) return;
  const int parts = fit_parts(f, sizeof(T) == 8);
  if (static_cast<int>(blockIdx.y) >= parts) return;
  double se = 0.0, sx = 0.0;
  fit_blocks<T>(fa, f, static_cast<const T*>(d.X), static_cast<const T*>(d.fitw), blockIdx.y,
                parts, fit_dyn, chain, slice, se, sx);
  fit_block_reduce(se, sx, red);
  if (threadIdx.x == 0) {
    d.fitp[blockIdx.y] = se;
    d.fitp[kFitParts + blockIdx.y] = sx;
  }
}

// Slots with FP32 X and K <= 128: the contraction on the tensor cores (fit_tc.cuh).
__global__ void __launch_bounds__(FNT, 1) kb_fit_tc(const BInst* __restrict__ tab,
                                                    unsigned* err) {
  extern __shared__ __align__(1024) unsigned char fit_tc_dyn[];
  __shared__ float chain[8][kMaxL];
  __shared__ float slice[8][kMaxL];
  __shared__ double red[2 * (FNT / 32)];
  __shared__ FitArgs fa;
  __shared__ FitTcShared sh;
  const BInst& d = tab[blockIdx.x];
  if (!fit_due(d) || d.xf64) return;
  if (threadIdx.x == 0) fit_args(d, fa);
  __syncthreads();
  const FitSplit f = fit_split(fa.N, fa.dims, fa.ranks);
  if (!fit_use_tc(f, false)) return;
  const int parts = fit_parts(f, false);
  if (static_cast<int>(blockIdx.y) >= parts) return;
  double se = 0.0, sx = 0.0;
  fit_tc_blocks(fa, f, static_cast<const float*>(d.X),
                static_cast<const unsigned char*>(d.fitw),
                blockIdx.y, parts, fit_tc_dyn, chain, slice, sh, err, se, sx);
  fit_block_reduce(se, sx, red);
  if (threadIdx.x == 0) {
    d.fitp[blockIdx.y] = se;
    d.fitp[kFitParts + blockIdx.y] = sx;
  }
}

__global__ void __launch_bounds__(128) kb_advance(const BInst* __restrict__ tab, int count,
                                                  int xf64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const BInst& d = tab[i];
  if (!d.slot) return;
  SlotState& s = *d.slot;
  if (s.status != kSlotRunning) return;
  const int t = s.step;
  if (t >= 0 && *d.info != 0) s.singular += 1;
  if (fit_due(d)) {
    const FitSplit f = fit_split(d.N, d.dims, d.ranks);
    const int parts = fit_parts(f, xf64 != 0);
    double se = 0.0, sx = 0.0;
    for (int q = 0; q < parts; ++q) {
      se += d.fitp[q];
      sx += d.fitp[kFitParts + q];
    }
    const double rel = sx > 0.0 ? sqrt(se / sx) : (se > 0.0 ? INFINITY : 0.0);
    const double fit = 1.0 - rel;
    const int sw = s.sweeps + 1;
    s.sweeps = sw;
    s.fit_prev = s.fit;
    s.fit = fit;
    if (sw <= kMaxServedSweeps) d.hist[sw - 1] = fit;
    if (!isfinite(fit)) s.status = kSlotFailed;
    else if (sw >= 2 && fabs(fit - s.fit_prev) < s.tol) s.status = kSlotConverged;
    else if (sw >= s.max_sweeps) s.status = kSlotCapped;
  }
  s.step = t + 1;
}

}  // namespace

cudaError_t bl_fit(const BLaunch& b, unsigned* err, cudaStream_t st) {
  dim3 rgrid(b.count, kFitRightCtas);
  dim3 grid(b.count, kFitParts);
  constexpr int kSplitK = 128;
  const int k_small = b.Lmax < kSplitK ? b.Lmax : kSplitK;
  if (b.xf64) {
    kb_fit_right<double><<<rgrid, FNT, 0, st>>>(b.tab);
    kb_fit<double><<<grid, FNT, fit_smem_bytes<double>(k_small), st>>>(b.tab, 0, kSplitK);
    if (b.Lmax > kSplitK)
      kb_fit<double><<<grid, FNT, fit_smem_bytes<double>(b.Lmax), st>>>(b.tab, kSplitK, kMaxL);
  } else {
    kb_fit_right<float><<<rgrid, FNT, 0, st>>>(b.tab);
    kb_fit_tc<<<grid, FNT, kFitTcSmem, st>>>(b.tab, err);
    if (b.Lmax > kFitTcMaxK)
      kb_fit<float><<<grid, FNT, fit_smem_bytes<float>(b.Lmax), st>>>(b.tab, kFitTcMaxK, kMaxL);
  }
  return cudaGetLastError();
}

cudaError_t bl_advance(const BLaunch& b, cudaStream_t st) {
  kb_advance<<<(b.count + 127) / 128, 128, 0, st>>>(b.tab, b.count, b.xf64 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t batched_fit_attributes() {
  cudaError_t e = cudaFuncSetAttribute(kb_fit<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(fit_smem_bytes<float>(kMaxL)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kb_fit_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kFitTcSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kb_fit<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(fit_smem_bytes<double>(kMaxL)));
}

}  // namespace trk
