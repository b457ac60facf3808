// Batched one-CTA Cholesky factorisations (cholesky_body.cuh): the normal matrix of each
// instance's LS step (Alg. 2) and the Grams of its leverage passes (Def. 4).
#include "batched_kern.cuh"
#include "cholesky_body.cuh"

namespace trk {
namespace {

// ------------------------------------------------------------------------------------
// Cholesky factorisations, one CTA per instance.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(CNT) kb_cholesky(const BInst* __restrict__ tab, int step,
                                                   int init_k, int which, unsigned* err,
                                                   int smem_bytes, int mixed, int ls_mode) {
  extern __shared__ double smem[];
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, which != 0);
  if (!cu.active) return;
  const double eps = 2.220446049250313e-16, eps32 = 1.1920928955078125e-07;
  const bool tall = cu.I >= cu.L;
  if (which == 0) {
    const int n = cu.L;
    const int64_t nn = static_cast<int64_t>(n) * n;
    double* A = (nn * 8 <= smem_bytes) ? smem : d.Lrow;
    if (mixed) {
      float* A32 = (nn * 4 <= smem_bytes) ? reinterpret_cast<float*>(smem)
                                          : reinterpret_cast<float*>(d.Lrow);
      cholesky_cta_mixed<float>(d.M, n, ls_mode, static_cast<double>(n) * eps,
                                static_cast<double>(n) * eps32, A32, A, d.Lrow, d.Lcol,
                                d.invdiag, d.keep, d.info, err, static_cast<float*>(d.limg),
                                d.mimg);
      return;
    }
    cholesky_cta(d.M, n, ls_mode, static_cast<double>(n) * eps, A, d.Lrow, d.Lcol, d.invdiag,
                 d.keep, d.info, err, static_cast<double*>(d.limg), nullptr, nullptr);
    return;
  }
  const double tol = static_cast<double>(cu.I > cu.L ? cu.I : cu.L) * eps;
  if (which == 1) {
    const int n = tall ? cu.L : static_cast<int>(cu.I);
    const int64_t nn = static_cast<int64_t>(n) * n;
    double* A = (nn * 8 <= smem_bytes) ? smem : d.L1row;
    if (mixed && tall) {   // double-float first; a wide pass-1 factor feeds pass 2 (FP64)
      const double eps_ff = 9.094947017729282e-13;   // 2^-40
      float* Aff = (panel_floats<FFOps>(n) * 4 <= smem_bytes) ? reinterpret_cast<float*>(smem)
                                                               : nullptr;
      cholesky_cta_lev_mixed(d.G1, n, tol, tol / eps * eps_ff, Aff, A, d.L1row, d.L1col, d.inv1,
                             d.keep1, d.info1, err, d.img1);
      return;
    }
    cholesky_cta(d.G1, n, 1, tol, A, d.L1row, d.L1col, d.inv1, d.keep1, d.info1, err, d.img1,
                 nullptr, nullptr);
    return;
  }
  if (tall) return;
  const int n = static_cast<int>(cu.I);
  double* A = (static_cast<int64_t>(n) * n * 8 <= smem_bytes) ? smem : d.L2row;
  cholesky_cta(d.G2, n, 1, tol, A, d.L2row, d.L2col, d.inv2, d.keep2, d.info2, err, d.img2,
               nullptr, nullptr);
}

// The FP64 image of a double-float leverage factor from the FP32 planes the factorisation
// left in L1row / L1col (*info1 == 2; tall mixed instances only).
__global__ void __launch_bounds__(256) kb_ff_image(const BInst* __restrict__ tab, int step,
                                                   int init_k) {
  const BInst& d = tab[blockIdx.x];
  const Cur cu = current(d, step, init_k, true);
  if (!cu.active || cu.I < cu.L || *d.info1 != 2) return;
  const int n = cu.L;
  const int64_t count = static_cast<int64_t>(n) * (n + 1);
  const float* hi = reinterpret_cast<const float*>(d.L1row);
  const float* lo = reinterpret_cast<const float*>(d.L1col);
  for (int64_t e = static_cast<int64_t>(blockIdx.y) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.y) * blockDim.x)
    d.img1[e] = static_cast<double>(hi[e]) + static_cast<double>(lo[e]);
}

int smem_for_cholesky(int nmax) {
  const int64_t need = static_cast<int64_t>(nmax) * nmax * 8;
  const int64_t ff = panel_floats<FFOps>(nmax) * 4;
  if ((ff > need ? ff : need) <= kDyn) return static_cast<int>(ff > need ? ff : need);
  return need <= kDyn ? static_cast<int>(need) : 0;
}

}  // namespace

cudaError_t bl_cholesky(const BLaunch& b, int step, int init_k, int which, unsigned* err,
                        cudaStream_t st) {
  const int nmax = which == 0 ? b.Lmax : (which == 1 ? b.n1max : b.n2max);
  if (nmax <= 0) return cudaSuccess;
  const int dyn = smem_for_cholesky(nmax);
  kb_cholesky<<<b.count, CNT, dyn, st>>>(b.tab, step, init_k, which, err, dyn, b.f64 ? 0 : 1,
                                          b.ls_mode);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || which != 1 || b.f64) return e;
  // double-float leverage factors leave FP32 planes: their FP64 image
  const int64_t count = static_cast<int64_t>(nmax) * (nmax + 1);
  dim3 grid(b.count, static_cast<unsigned>((count + 255) / 256 < 16 ? (count + 255) / 256 : 16));
  kb_ff_image<<<grid, 256, 0, st>>>(b.tab, step, init_k);
  return cudaGetLastError();
}

cudaError_t batched_chol_attributes() {
  return cudaFuncSetAttribute(kb_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, kDyn);
}

}  // namespace trk
