// Row a6, mixed-precision LS step for L <= 128: the solve of M Z = B (M = L_f L_f^T from the
// FP32 or FP64 factorisation, FP32 image) with one step of iterative refinement, as
//   W = L_f^-1 (explicit, FP32);  z = W^T W b;  r = b - M z;  z += W^T W r,
// the same arithmetic structure as the substitution kernel's mode 2 (two substitutions, the
// residual against M's FP32 image, two more substitutions), with each substitution turned
// into a product by W. W normally comes with the factor from the one-CTA factor-and-inverse
// pass (chol_inv.cuh); after its fallback factorisation, k_tri_inv forms it with one
// triangular solve per column, many warps in parallel. The solves of the I right-hand sides are then
// small dense products (k_solve_inv), which spread over the GPU instead of running one
// 100-step dependent chain per warp. A dropped column (inverse pivot 0) gives a zero row and
// column of W, so its unknown is 0 and it updates nothing, as in the substitutions.
#include "common.cuh"

namespace trk {
namespace {

constexpr int IW = 4;          // warps per CTA of the inverse
constexpr int SNT = 128;       // threads per CTA of the solve
constexpr int SNR = 4;         // right-hand sides per CTA of the solve

__device__ __forceinline__ void stage16(void* dst, const void* src, int bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const char* s = static_cast<const char*>(src);
  for (int o = threadIdx.x * 16; o < bytes; o += blockDim.x * 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d + o), "l"(s + o) : "memory");
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__host__ __device__ inline int img_bytes32(int n) { return ((n * (n + 1) * 4 + 15) / 16) * 16; }

// Column j of W = L^-1 by forward substitution of e_j, one warp per column; lane l holds rows
// l, l+32, .. (QN registers). W is written as the padded column-major image W[j*(n+1) + r].
template <int QN>
__global__ void __launch_bounds__(IW * 32) k_tri_inv(int n, const float* __restrict__ Limg,
                                                     const double* __restrict__ invdiag,
                                                     const int* __restrict__ info,
                                                     float* __restrict__ Wimg,
                                                     const int* __restrict__ skip_if) {
  extern __shared__ __align__(16) unsigned char ism[];
  if (*info != 0 || (skip_if && *skip_if)) return;
  const int np = n + 1;
  float* inv = reinterpret_cast<float*>(ism);
  float* Ls = inv + kMaxL;
  stage16(Ls, Limg, img_bytes32(n));
  for (int c = threadIdx.x; c < n; c += blockDim.x) inv[c] = static_cast<float>(invdiag[c]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * IW + warp;
  if (j >= n) return;
  float x[QN];
#pragma unroll
  for (int q = 0; q < QN; ++q) x[q] = (lane + 32 * q == j) ? 1.0f : 0.0f;
  for (int qb = j >> 5; qb < QN; ++qb) {
    float xb = x[0];
#pragma unroll
    for (int q = 1; q < QN; ++q) xb = (q == qb) ? x[q] : xb;
#pragma unroll
    for (int lc = 0; lc < 32; ++lc) {
      const int c = qb * 32 + lc;
      if (c >= n) break;
      if (c < j) continue;
      const float xc = __shfl_sync(0xffffffffu, xb, lc) * inv[c];
      if (lane == lc) xb = xc;
      if (lane > lc && qb * 32 + lane < n) xb = fmaf(-Ls[c * np + qb * 32 + lane], xc, xb);
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        if (q > qb) {
          const int r = lane + 32 * q;
          if (r < n) x[q] = fmaf(-Ls[c * np + r], xc, x[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < QN; ++q)
      if (q == qb) x[q] = xb;
  }
#pragma unroll
  for (int q = 0; q < QN; ++q) {
    const int r = lane + 32 * q;
    if (r < n) Wimg[j * np + r] = r >= j ? x[q] : 0.0f;
  }
}

// y = W x (lower triangular; W[r][c] = Ws[c*np + r]) for SNR vectors of length n in shared
// memory (x[c*SNR + v]); thread t < n computes row t.
__device__ __forceinline__ void lower_mv(const float* Ws, int n, int np, const float* x,
                                         float* y) {
  const int r = threadIdx.x;
  if (r < n) {
    float acc[SNR] = {};
    for (int c = 0; c <= r; ++c) {
      const float w = Ws[c * np + r];
      const float4 xv = *reinterpret_cast<const float4*>(x + c * SNR);
      acc[0] = fmaf(w, xv.x, acc[0]);
      acc[1] = fmaf(w, xv.y, acc[1]);
      acc[2] = fmaf(w, xv.z, acc[2]);
      acc[3] = fmaf(w, xv.w, acc[3]);
    }
    *reinterpret_cast<float4*>(y + r * SNR) = make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
}

// y = W^T x (upper triangular: y_c = sum_{r >= c} W[r][c] x_r); thread t < n computes row t.
__device__ __forceinline__ void upper_mv(const float* Ws, int n, int np, const float* x,
                                         float* y) {
  const int c = threadIdx.x;
  if (c < n) {
    float acc[SNR] = {};
    for (int r = c; r < n; ++r) {
      const float w = Ws[c * np + r];
      const float4 xv = *reinterpret_cast<const float4*>(x + r * SNR);
      acc[0] = fmaf(w, xv.x, acc[0]);
      acc[1] = fmaf(w, xv.y, acc[1]);
      acc[2] = fmaf(w, xv.z, acc[2]);
      acc[3] = fmaf(w, xv.w, acc[3]);
    }
    *reinterpret_cast<float4*>(y + c * SNR) = make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
}

// SNR right-hand sides per CTA (b = row v of B^T): z = W^T W b, r = b - M z, z += W^T W r,
// then core_out[v][a][b] = z[a + Rl*b].
__global__ void __launch_bounds__(SNT) k_solve_inv(int n, const float* __restrict__ Wimg,
                                                   const float* __restrict__ Mimg,
                                                   const int* __restrict__ info, int64_t nvec,
                                                   const double* __restrict__ rhs, int64_t ld,
                                                   int Rl, int Rr, double* __restrict__ core_out) {
  extern __shared__ __align__(16) unsigned char ssm[];
  if (*info != 0) return;
  const int np = n + 1;
  const int ib = img_bytes32(n);
  float* Ws = reinterpret_cast<float*>(ssm);
  float* Ms = reinterpret_cast<float*>(ssm + ib);
  float* b = reinterpret_cast<float*>(ssm + 2 * ib);    // [n][SNR]
  float* t = b + kMaxL * SNR;
  float* z = t + kMaxL * SNR;
  const int64_t v0 = static_cast<int64_t>(blockIdx.x) * SNR;
  for (int e = threadIdx.x; e < n * SNR; e += SNT) {
    const int r = e / SNR, v = e % SNR;
    b[e] = (v0 + v < nvec) ? static_cast<float>(rhs[(v0 + v) * ld + r]) : 0.0f;
  }
  stage16(Ws, Wimg, ib);
  stage16(Ms, Mimg, ib);
  __syncthreads();
  lower_mv(Ws, n, np, b, t);
  __syncthreads();
  upper_mv(Ws, n, np, t, z);
  __syncthreads();
  // residual r = b - M z into t (M symmetric: M[r][c] = Ms[c*np + r])
  if (threadIdx.x < n) {
    const int r = threadIdx.x;
    float acc[SNR];
#pragma unroll
    for (int v = 0; v < SNR; ++v) acc[v] = b[r * SNR + v];
    for (int c = 0; c < n; ++c) {
      const float m = Ms[c * np + r];
      const float4 zv = *reinterpret_cast<const float4*>(z + c * SNR);
      acc[0] = fmaf(-m, zv.x, acc[0]);
      acc[1] = fmaf(-m, zv.y, acc[1]);
      acc[2] = fmaf(-m, zv.z, acc[2]);
      acc[3] = fmaf(-m, zv.w, acc[3]);
    }
    *reinterpret_cast<float4*>(t + r * SNR) = make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
  __syncthreads();
  lower_mv(Ws, n, np, t, b);     // b is free now
  __syncthreads();
  upper_mv(Ws, n, np, b, t);
  __syncthreads();
  for (int e = threadIdx.x; e < n * SNR; e += SNT) {
    const int r = e / SNR, v = e % SNR;
    if (v0 + v < nvec) {
      const int a = r % Rl, bb = r / Rl;
      core_out[(v0 + v) * n + a * Rr + bb] = static_cast<double>(z[e] + t[e]);
    }
  }
}

size_t inv_smem(int n) { return kMaxL * 4 + img_bytes32(n); }
size_t solve_smem_bytes(int n) { return 2 * img_bytes32(n) + 3 * kMaxL * SNR * 4; }

}  // namespace

bool solve_inv_fits(int n) { return n >= 1 && n <= 128; }

size_t solve_inv_workspace(int n) { return img_bytes32(n); }

cudaError_t launch_solve_inv(int n, const float* Limg, const float* Mimg,
                             const double* invdiag, const int* info, int64_t nvec,
                             const double* rhs, int64_t ld, int Rl, int Rr, double* core_out,
                             float* Wimg, cudaStream_t st, const int* fast) {
  if (!solve_inv_fits(n)) return cudaErrorInvalidValue;
  if (nvec <= 0) return cudaSuccess;
  const unsigned ib = static_cast<unsigned>((n + IW - 1) / IW);
  switch ((n + 31) / 32) {
    case 1: k_tri_inv<1><<<ib, IW * 32, inv_smem(n), st>>>(n, Limg, invdiag, info, Wimg, fast); break;
    case 2: k_tri_inv<2><<<ib, IW * 32, inv_smem(n), st>>>(n, Limg, invdiag, info, Wimg, fast); break;
    case 3: k_tri_inv<3><<<ib, IW * 32, inv_smem(n), st>>>(n, Limg, invdiag, info, Wimg, fast); break;
    default: k_tri_inv<4><<<ib, IW * 32, inv_smem(n), st>>>(n, Limg, invdiag, info, Wimg, fast); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned sb = static_cast<unsigned>((nvec + SNR - 1) / SNR);
  k_solve_inv<<<sb, SNT, solve_smem_bytes(n), st>>>(n, Wimg, Mimg, info, nvec, rhs, ld, Rl, Rr,
                                                     core_out);
  return cudaGetLastError();
}

cudaError_t solve_inv_attributes() {
  const int di = static_cast<int>(inv_smem(128)), ds = static_cast<int>(solve_smem_bytes(128));
  cudaError_t e = cudaFuncSetAttribute(k_tri_inv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, di);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tri_inv<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, di);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tri_inv<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, di);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tri_inv<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, di);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_solve_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, ds);
  return e;
}

}  // namespace trk
