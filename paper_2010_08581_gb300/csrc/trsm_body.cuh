// Triangular solves with a Cholesky factor L (n <= 256) for many vectors, shared by the
// single-problem kernel (trsm.cu) and the batched kernel (batched.cu):
//   mode 0 (leverage rows, row a1): ell_v = || L^-1 a_v ||^2 -- row norms of Q = A R^-1 of
//           the Cholesky-based thin QR (Def. 4), optionally followed by p and the CDF;
//   mode 1 (LS solve, row a6):      z_v = L^-T L^-1 b_v, written into the new core;
//   mode 2 (LS solve + one refinement step, row a6):
//           z = L^-T L^-1 b;  r = b - M z;  z += L^-T L^-1 r.
// One warp owns NB vectors; lane l holds rows l, l+32, ... (QN registers per vector), so a
// substitution step is one shuffle broadcast plus independent FMAs. The factor (and M) are
// staged in shared memory with a padded row stride (n+1): from the padded images written
// by the Cholesky kernel (cp.async, 16 bytes per request) when given, else converted from
// the FP64 column-major factor.
#pragma once

#include "common.cuh"

namespace trk {

constexpr int TW = 4;   // warps per CTA

// The factor for the substitutions: the padded image s[c*(n+1) + r] = L[r][c] in shared
// memory (SMEM), or in global memory when the Cholesky kernel wrote one (its FP32 or FP64
// image in L2: no per-element conversion from FP64), else the FP64 column- and row-major
// factor.
// PACK (with SMEM): the lower triangle packed column by column in shared memory, column c
// starting at c*n - c(c-1)/2 -- for factors whose padded image does not fit (n > 160 in
// FP32): n(n+1)/2 entries.
template <typename T, bool SMEM, bool PACK = false>
struct Factor {
  const T* s;            // image, shared (SMEM) or global (gimg)
  const double* Lcol;    // global: Lcol[c*n + r] = L[r][c]
  const double* Lrow;    // global: Lrow[c*n + r] = L[c][r]
  int n;
  bool gimg = false;     // !SMEM: s is a global image
  __device__ __forceinline__ int pk(int c) const { return c * n - (c * (c - 1)) / 2 - c; }
  __device__ __forceinline__ T col(int c, int r) const {   // L[r][c], r >= c
    if constexpr (PACK) return s[pk(c) + r];
    else if constexpr (SMEM) return s[c * (n + 1) + r];
    else return gimg ? __ldg(s + c * (n + 1) + r) : static_cast<T>(Lcol[c * n + r]);
  }
  __device__ __forceinline__ T row(int c, int r) const {   // L[c][r], r < c
    if constexpr (PACK) return s[pk(r) + c];
    else if constexpr (SMEM) return s[r * (n + 1) + c];
    else return gimg ? __ldg(s + r * (n + 1) + c) : static_cast<T>(Lrow[c * n + r]);
  }
};

template <typename T, int QN, int NB>
__device__ __forceinline__ T pick(const T (&x)[QN][NB], int q, int v) {
  T s = x[0][v];
#pragma unroll
  for (int u = 1; u < QN; ++u) s = (u == q) ? x[u][v] : s;
  return s;
}

template <typename T, int QN, int NB>
__device__ __forceinline__ void put(T (&x)[QN][NB], int q, int v, T val) {
#pragma unroll
  for (int u = 0; u < QN; ++u)
    if (u == q) x[u][v] = val;
}

// x <- L^-1 x. Rows are processed in blocks of 32 (register slot qb of every lane); inside a
// block the pivot row's lane is a compile-time constant and the block's values live in one
// register per vector, so one step is a shuffle, a multiply and independent FMAs.
template <typename T, int QN, int NB, bool SMEM, bool PACK>
__device__ __forceinline__ void forward(T (&x)[QN][NB], const Factor<T, SMEM, PACK>& F,
                                        const T* inv, int lane) {
  const int n = F.n;
  for (int qb = 0; qb < QN; ++qb) {
    T xb[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) xb[v] = pick(x, qb, v);
#pragma unroll
    for (int lc = 0; lc < 32; ++lc) {
      const int c = qb * 32 + lc;
      if (c >= n) break;
      const T ic = inv[c];
      T xc[NB];
#pragma unroll
      for (int v = 0; v < NB; ++v) {
        xc[v] = __shfl_sync(0xffffffffu, xb[v], lc) * ic;
        if (lane == lc) xb[v] = xc[v];
      }
      if (lane > lc && qb * 32 + lane < n) {
        const T l = F.col(c, qb * 32 + lane);
#pragma unroll
        for (int v = 0; v < NB; ++v) xb[v] -= l * xc[v];
      }
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        if (q > qb) {
          const int r = lane + 32 * q;
          const T l = (r < n) ? F.col(c, r) : T(0);
#pragma unroll
          for (int v = 0; v < NB; ++v) x[q][v] -= l * xc[v];
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NB; ++v) put(x, qb, v, xb[v]);
  }
}

// x <- L^-T x, blocks in reverse order.
template <typename T, int QN, int NB, bool SMEM, bool PACK>
__device__ __forceinline__ void backward(T (&x)[QN][NB], const Factor<T, SMEM, PACK>& F,
                                         const T* inv, int lane) {
  const int n = F.n;
  for (int qb = QN - 1; qb >= 0; --qb) {
    T xb[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) xb[v] = pick(x, qb, v);
#pragma unroll
    for (int lc = 31; lc >= 0; --lc) {
      const int c = qb * 32 + lc;
      if (c >= n) continue;
      const T ic = inv[c];
      T zc[NB];
#pragma unroll
      for (int v = 0; v < NB; ++v) {
        zc[v] = __shfl_sync(0xffffffffu, xb[v], lc) * ic;
        if (lane == lc) xb[v] = zc[v];
      }
      if (lane < lc) {
        const T l = F.row(c, qb * 32 + lane);
#pragma unroll
        for (int v = 0; v < NB; ++v) xb[v] -= l * zc[v];
      }
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        if (q < qb) {
          const T l = F.row(c, lane + 32 * q);
#pragma unroll
          for (int v = 0; v < NB; ++v) x[q][v] -= l * zc[v];
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NB; ++v) put(x, qb, v, xb[v]);
  }
}

// Copy `bytes` (multiple of 16) from global to shared memory with cp.async, all threads.
__device__ __forceinline__ void stage_async(void* dst, const void* src, int bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const char* s = static_cast<const char*>(src);
  for (int o = threadIdx.x * 16; o < bytes; o += blockDim.x * 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d + o), "l"(s + o) : "memory");
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Block-wide exclusive scan (fixed order) of one double per thread for NW warps.
template <int NW>
__device__ __forceinline__ double block_scan_nw(double v, double* wt, double* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wt[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0.0;
    for (int q = 0; q < NW; ++q) { const double t = wt[q]; wt[q] = run; run += t; }
    *total = run;
  }
  __syncthreads();
  const double r = wt[warp] + inc - v;
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_scan_tw(double v, double* wt, double* total) {
  return block_scan_nw<TW>(v, wt, total);
}

// p = ell / sum(ell) and its prefix sum, by the CTA that finishes last (mode 0 only), whose
// NW warps all take part.
template <int NW>
__device__ inline void cdf_epilogue_nw(const CdfEpilogue& ep, const double* ell, int64_t I) {
  __shared__ double wt[NW];
  __shared__ double s_total;
  if (ep.skip && *ep.skip) return;
  const int t = threadIdx.x;
  const int64_t chunk = (I + NW * 32 - 1) / (NW * 32);
  const int64_t b = t * chunk, e = (b + chunk < I) ? b + chunk : I;
  double s = 0.0;
  for (int64_t i = b; i < e; ++i) s += __ldcg(ell + i);
  block_scan_nw<NW>(s, wt, &s_total);
  const double total = s_total;
  if (!(total > 0.0) || !isfinite(total)) {
    for (int64_t i = b; i < e; ++i) {
      ep.p[i] = 1.0 / static_cast<double>(I);
      ep.cdf[i] = static_cast<double>(i + 1) / static_cast<double>(I);
    }
    if (t == 0) atomicOr(ep.err, kErrSingular);
    return;
  }
  // one division: p_i = ell_i * (1 / total) (within an ulp of ell_i / total; an FP64 division
  // per entry costs far more than the multiply on this GPU's FP64 pipe)
  const double rt = 1.0 / total;
  double sp = 0.0;
  for (int64_t i = b; i < e; ++i) sp += __ldcg(ell + i) * rt;
  double run = block_scan_nw<NW>(sp, wt, &s_total);
  for (int64_t i = b; i < e; ++i) {
    const double pi = __ldcg(ell + i) * rt;
    ep.p[i] = pi;
    run += pi;
    ep.cdf[i] = run;
  }
}

__device__ inline void cdf_epilogue(const CdfEpilogue& ep, const double* ell, int64_t I) {
  cdf_epilogue_nw<TW>(ep, ell, I);
}

template <typename T, int QN, int NB, bool SMEM, bool PACK = false>
__device__ __forceinline__ void trsm_cta(unsigned char* trsm_smem, int64_t cta, int n,
                                         const double* __restrict__ Lrow,
                                                  const double* __restrict__ Lcol,
                                                  const double* __restrict__ invdiag,
                                                  const int* __restrict__ info, int64_t nvec,
                                                  const double* __restrict__ rhs, int64_t ld,
                                                  int mode, const double* __restrict__ M,
                                                  const T* __restrict__ Limg,
                                                  const float* __restrict__ Mimg, int Rl, int Rr,
                                                  double* __restrict__ core_out,
                                                  double* __restrict__ ell, CdfEpilogue ep,
                                                  int nctas) {
  if ((info && *info) || (ep.run_if && *ep.run_if == 0)) return;
  const int np = n + 1;
  const int img_elems = ((n * np * static_cast<int>(sizeof(T)) + 15) / 16) * 16 /
                        static_cast<int>(sizeof(T));
  T* inv = reinterpret_cast<T*>(trsm_smem);                  // kMaxL entries
  T* Ls = inv + kMaxL;                                       // n*(n+1) (padded to 16 B)
  T* Ms = Ls + (SMEM && !PACK ? img_elems : 0);              // mode 2
  for (int c = threadIdx.x; c < n; c += blockDim.x) inv[c] = static_cast<T>(invdiag[c]);
  if constexpr (PACK) {
    // the lower triangle, column by column, from the padded image with element-sized
    // asynchronous copies (all in flight at once), or converted from the FP64 factor
    for (int c = threadIdx.x >> 5; c < n; c += TW) {
      const int base = c * n - (c * (c - 1)) / 2 - c;
      for (int r = c + (threadIdx.x & 31); r < n; r += 32) {
        if (Limg) {
          const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(Ls + base + r));
          if constexpr (sizeof(T) == 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d),
                         "l"(Limg + c * np + r) : "memory");
          else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d),
                         "l"(Limg + c * np + r) : "memory");
        } else {
          Ls[base + r] = static_cast<T>(Lcol[c * n + r]);
        }
      }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  } else if constexpr (SMEM) {
    if (Limg) {
      stage_async(Ls, Limg, img_elems * static_cast<int>(sizeof(T)));
    } else {
      for (int c = threadIdx.x >> 5; c < n; c += TW)
        for (int r = threadIdx.x & 31; r < n; r += 32) Ls[c * np + r] = static_cast<T>(Lcol[c * n + r]);
    }
    if (mode == 2) {
      if (Mimg && sizeof(T) == 4) {
        stage_async(Ms, Mimg, img_elems * static_cast<int>(sizeof(T)));
      } else {
        for (int c = threadIdx.x >> 5; c < n; c += TW)
          for (int r = threadIdx.x & 31; r < n; r += 32) Ms[c * np + r] = static_cast<T>(M[c * n + r]);
      }
    }
  }
  __syncthreads();
  Factor<T, SMEM, PACK> F{SMEM ? Ls : Limg, Lcol, Lrow, n, !SMEM && Limg != nullptr};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t v0 = (cta * TW + warp) * NB;
  if (mode == 0) {
    if (v0 < nvec) {
      T x[QN][NB];
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        const int r = lane + 32 * q;
#pragma unroll
        for (int v = 0; v < NB; ++v)
          x[q][v] = (r < n && v0 + v < nvec) ? static_cast<T>(rhs[(v0 + v) * ld + r]) : T(0);
      }
      forward(x, F, inv, lane);
#pragma unroll
      for (int v = 0; v < NB; ++v) {
        T s = T(0);
#pragma unroll
        for (int q = 0; q < QN; ++q)
          if (lane + 32 * q < n) s += x[q][v] * x[q][v];   // rows >= n hold no data
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && v0 + v < nvec) ell[v0 + v] = static_cast<double>(s);
      }
    }
    if (ep.counter) {      // the last CTA to finish forms p and the CDF
      __shared__ int s_last;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(ep.counter, 1u) == static_cast<unsigned>(nctas) - 1) ? 1 : 0;
      __syncthreads();
      if (s_last) {
        __threadfence();
        cdf_epilogue(ep, ell, nvec);
        if (threadIdx.x == 0) *ep.counter = 0u;
      }
    }
    return;
  }
  if (v0 >= nvec) return;
  T x[QN][NB];
#pragma unroll
  for (int q = 0; q < QN; ++q) {
    const int r = lane + 32 * q;
#pragma unroll
    for (int v = 0; v < NB; ++v)
      x[q][v] = (r < n && v0 + v < nvec) ? static_cast<T>(rhs[(v0 + v) * ld + r]) : T(0);
  }
  forward(x, F, inv, lane);
  backward(x, F, inv, lane);
  if (mode == 2) {
    // residual r = b - M z (M symmetric: column t of M = row t)
    T res[QN][NB];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int r = lane + 32 * q;
#pragma unroll
      for (int v = 0; v < NB; ++v)
        res[q][v] = (r < n && v0 + v < nvec) ? static_cast<T>(rhs[(v0 + v) * ld + r]) : T(0);
    }
    for (int qt = 0; qt < QN; ++qt) {
      T xt[NB];
#pragma unroll
      for (int v = 0; v < NB; ++v) xt[v] = pick(x, qt, v);
#pragma unroll 8
      for (int lt = 0; lt < 32; ++lt) {
        const int t = qt * 32 + lt;
        if (t >= n) break;
        T zt[NB];
#pragma unroll
        for (int v = 0; v < NB; ++v) zt[v] = __shfl_sync(0xffffffffu, xt[v], lt);
#pragma unroll
        for (int q = 0; q < QN; ++q) {
          const int r = lane + 32 * q;
          if (r < n) {
            T m;
            if constexpr (SMEM && !PACK) m = Ms[t * np + r];
            else if (sizeof(T) == 4 && Mimg) m = static_cast<T>(__ldg(Mimg + t * np + r));
            else m = static_cast<T>(M[t * n + r]);
#pragma unroll
            for (int v = 0; v < NB; ++v) res[q][v] -= m * zt[v];
          }
        }
      }
    }
    forward(res, F, inv, lane);
    backward(res, F, inv, lane);
#pragma unroll
    for (int q = 0; q < QN; ++q)
#pragma unroll
      for (int v = 0; v < NB; ++v) x[q][v] += res[q][v];
  }
  // new core: core[i][a][b] = z[a + Rl*b]
#pragma unroll
  for (int q = 0; q < QN; ++q) {
    const int r = lane + 32 * q;
    if (r >= n) continue;
    const int a = r % Rl, b = r / Rl;
#pragma unroll
    for (int v = 0; v < NB; ++v)
      if (v0 + v < nvec) core_out[(v0 + v) * n + a * Rr + b] = static_cast<double>(x[q][v]);
  }
}


// Shared memory of the packed layout (the inverse diagonal and n(n+1)/2 factor entries).
template <typename T>
__host__ __device__ inline size_t packed_bytes(int n) {
  return kMaxL * sizeof(T) +
         ((static_cast<size_t>(n) * (n + 1) / 2 * sizeof(T) + 15) / 16) * 16;
}

template <typename T>
__host__ __device__ inline size_t staged_bytes(int n, int mode) {
  const size_t img = ((static_cast<size_t>(n) * (n + 1) * sizeof(T) + 15) / 16) * 16;
  return kMaxL * sizeof(T) + (mode == 2 ? 2 : 1) * img;
}

}  // namespace trk
