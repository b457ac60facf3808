// Row a1 for wide unfoldings (I < L): leverage scores of the rows of an I x L matrix A by
// one-sided Jacobi (Hestenes, 1958) in FP64, and from them p^(n) and its CDF (Def. 4; eq. for
// p^(n)).
//
// The rows b_0 .. b_{I-1} of B = V^T A (V orthogonal, starting from B = A, V = I) are
// rotated in pairs until they are mutually orthogonal: then A = V B with B B^T diagonal, so
// V holds the left singular vectors of A and ||b_k|| its singular values. The rank rule is
// the one a singular value decomposition applies: sigma_k > max(I, L) * eps * sigma_max.
// The leverage score of row i is sum over the kept k of V[i][k]^2. Orthogonal rotations keep
// the backward error at a few eps * ||A||, so singular values far below sqrt(eps) sigma_max
// are resolved (a Gram matrix would square them away).
//
// One CTA per matrix: A (copied to shared memory) and V stay on chip. Pairs follow the
// round-robin (circle) order: in each of the I'-1 rounds (I' = I rounded up to even) the I'/2
// disjoint pairs are rotated by separate warps, one pair per warp at a time; a lane holds
// every 32nd column of the pair's two rows. Sweeps repeat until one makes no rotation (at
// most kMaxSweeps). Sums are in a fixed order, so the result does not depend on timing.
#include "common.cuh"

namespace trk {
namespace {

constexpr int JT = 256;            // threads per CTA
constexpr int JW = JT / 32;
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pair k of round r of the circle method on n (even) players: player n-1 stays fixed.
__device__ __forceinline__ void round_pair(int n, int r, int k, int* p, int* q) {
  const int m = n - 1;
  if (k == 0) {
    *p = m;
    *q = r;
  } else {
    *p = (r + k) % m;
    *q = (r - k + m) % m;
  }
}

__global__ void __launch_bounds__(JT) k_leverage_jacobi(const double* __restrict__ A, int I,
                                                        int L, int64_t lda,
                                                        double* __restrict__ ell,
                                                        double* __restrict__ p,
                                                        double* __restrict__ cdf,
                                                        const int* __restrict__ skip,
                                                        unsigned* err) {
  extern __shared__ __align__(16) double jsm[];
  const int n = I + (I & 1);            // even player count; a padded row stays zero
  double* B = jsm;                      // [n][L]
  double* V = B + static_cast<int64_t>(n) * L;   // [n][n], V[i][k] at i*n + k
  double* sig = V + static_cast<int64_t>(n) * n;  // [n]
  __shared__ int s_rot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int64_t e = tid; e < static_cast<int64_t>(n) * L; e += JT) {
    const int i = static_cast<int>(e / L), c = static_cast<int>(e - static_cast<int64_t>(i) * L);
    B[e] = i < I ? A[static_cast<int64_t>(i) * lda + c] : 0.0;
  }
  for (int e = tid; e < n * n; e += JT) V[e] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();
  const double rot_tol = 4.0 * 2.220446049250313e-16;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < n - 1; ++r) {
      for (int k = warp; k < n / 2; k += JW) {
        int a, b;
        round_pair(n, r, k, &a, &b);
        if (a > b) { const int t = a; a = b; b = t; }
        double* ra = B + static_cast<int64_t>(a) * L;
        double* rb = B + static_cast<int64_t>(b) * L;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int c = lane; c < L; c += 32) {
          const double x = ra[c], y = rb[c];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al == 0.0 || be == 0.0 || !(fabs(ga) > rot_tol * sqrt(al * be))) continue;
        // rotation zeroing the inner product of rows a and b
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int c = lane; c < L; c += 32) {
          const double x = ra[c], y = rb[c];
          ra[c] = cs * x - sn * y;
          rb[c] = sn * x + cs * y;
        }
        for (int i = lane; i < n; i += 32) {
          const double x = V[i * n + a], y = V[i * n + b];
          V[i * n + a] = cs * x - sn * y;
          V[i * n + b] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rotated = s_rot;
    __syncthreads();
    if (!rotated) break;
  }
  // singular values: the row norms of B
  for (int k = warp; k < n; k += JW) {
    const double* rk = B + static_cast<int64_t>(k) * L;
    double s = 0.0;
    for (int c = lane; c < L; c += 32) s = fma(rk[c], rk[c], s);
    s = warp_sum(s);
    if (lane == 0) sig[k] = sqrt(s);
  }
  __syncthreads();
  if (warp == 0) {
    double smax = 0.0;
    for (int k = 0; k < I; ++k) smax = fmax(smax, sig[k]);
    const double thr = static_cast<double>(I > L ? I : L) * 2.220446049250313e-16 * smax;
    // ell_i = sum over kept k of V[i][k]^2 (k in index order)
    for (int i = lane; i < I; i += 32) {
      double s = 0.0;
      for (int k = 0; k < I; ++k)
        if (sig[k] > thr) s = fma(V[i * n + k], V[i * n + k], s);
      ell[i] = s;
    }
    __syncwarp();
    if (lane == 0 && !(skip && *skip != 0)) {
      double tot = 0.0;
      for (int i = 0; i < I; ++i) tot += ell[i];
      if (!(tot > 0.0)) {
        if (err) atomicOr(err, kErrSingular);   // zero matrix: uniform distribution
        double c = 0.0;
        for (int i = 0; i < I; ++i) {
          p[i] = 1.0 / static_cast<double>(I);
          c += p[i];
          cdf[i] = c;
        }
      } else {
        double c = 0.0;
        for (int i = 0; i < I; ++i) {
          p[i] = ell[i] / tot;
          c += p[i];
          cdf[i] = c;
        }
      }
    }
  }
}

}  // namespace

size_t leverage_jacobi_smem(int64_t I, int L) {
  const int64_t n = I + (I & 1);
  return static_cast<size_t>(n * L + n * n + n) * sizeof(double);
}

bool leverage_jacobi_fits(int64_t I, int L) {
  return I >= 1 && I < L && I <= kJacobiMaxI && leverage_jacobi_smem(I, L) <= kJacobiSmem;
}

cudaError_t launch_leverage_jacobi(const double* A, int64_t I, int L, int64_t lda, double* ell,
                                   double* p, double* cdf, const int* skip, unsigned* err,
                                   cudaStream_t st) {
  if (!leverage_jacobi_fits(I, L)) return cudaErrorInvalidValue;
  k_leverage_jacobi<<<1, JT, leverage_jacobi_smem(I, L), st>>>(
      A, static_cast<int>(I), L, lda, ell, p, cdf, skip, err);
  return cudaGetLastError();
}

cudaError_t jacobi_attributes() {
  return cudaFuncSetAttribute(k_leverage_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kJacobiSmem));
}

}  // namespace trk
