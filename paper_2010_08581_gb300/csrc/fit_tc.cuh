// The relative-error contraction of fit_body.cuh on the 5th-generation tensor cores, for
// X in FP32 and contraction length K <= 128.
//
// Per block of 128 rows the CTA forms V (the left slice products, one warp per row), splits
// every entry into TF32 parts hi = rna(v), lo = rna(v - hi) and keeps both, K-major and
// 128-byte swizzled, in shared memory for the whole block. For every tile of 128 columns
// the K chunks (32 wide) of W^T stream through two shared-memory stages, split the same way;
// one elected thread issues hi*hi + hi*lo + lo*hi per 8-wide k-step into one FP32
// accumulator in tensor memory (about FP32 accuracy), committing each chunk to the stage's
// mbarrier. The epilogue reads TR(p, q) back from tensor memory (warp w: rows 32 (w % 4)..,
// columns 64 (w / 4)..), forms (X - TR)^2 and X^2 in FP32 per tile and adds them to FP64
// per-thread totals. Every mbarrier wait is bounded: on expiry the CTA records the timeout
// bit, waits (bounded) for its issued MMAs, frees its tensor memory and stops.
#pragma once

#include "fit_body.cuh"
#include "tc_common.cuh"

namespace trk {

constexpr int kFitTcMaxK = 128;
constexpr int FTM = 128;                          // rows per block (MMA M)
constexpr int FTN = 128;                          // columns per tile (MMA N)
constexpr int FTK = 32;                           // K per chunk (one 128-byte swizzle row)
constexpr int FT_TILE = FTM * FTK * 4;            // 16 KB: hi or lo of one operand chunk
constexpr int FT_VBYTES = 2 * (kFitTcMaxK / FTK) * FT_TILE;   // V hi/lo, all chunks
constexpr int FT_STAGE = 2 * FT_TILE;             // W chunk hi + lo
constexpr size_t kFitTcSmem = FT_VBYTES + 2 * FT_STAGE + 1024;

// The tensor-core contraction serves FP32 X with K <= 128; the rest uses fit_blocks.
__host__ __device__ inline bool fit_use_tc(const FitSplit& f, bool xf64) {
  return !xf64 && f.K <= kFitTcMaxK;
}

__host__ __device__ inline int64_t fit_row_blocks(const FitSplit& f, bool xf64) {
  const int64_t rb = fit_use_tc(f, xf64) ? FTM : (xf64 ? FitTile<double>::FL : FitTile<float>::FL);
  return (f.rows + rb - 1) / rb;
}

struct FitTcShared {
  uint64_t mbar[2];
  uint32_t tmem_slot;
  int abort;
};

// Accumulates (se, sx) over the row blocks first, first + stride, ... All threads of the CTA
// call it; `dyn` holds kFitTcSmem bytes of dynamic shared memory.
__device__ inline void fit_tc_blocks(const FitArgs& a, const FitSplit& f,
                                     const float* __restrict__ X, const float* __restrict__ WT,
                                     int64_t first, int64_t stride, unsigned char* dyn,
                                     float (*chain)[kMaxL], float (*slice)[kMaxL],
                                     FitTcShared& sh, unsigned* err, double& se, double& sx) {
  using namespace tc;
  constexpr uint32_t kIdesc = idesc_tf32(FTM, FTN);
  constexpr uint32_t kTmemCols = FTN;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  unsigned char* vt = base;                 // chunk c: hi at c * 2 * FT_TILE, lo after it
  unsigned char* stg = base + FT_VBYTES;    // stage s: hi at s * FT_STAGE, lo after it
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = f.K, Kc = (K + FTK - 1) / FTK;
  const int Rlast = a.ranks[a.N - 1];

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&sh.tmem_slot)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(&sh.mbar[0]), 1);
    mbar_init(smem_u32(&sh.mbar[1]), 1);
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem_slot;
  long long gc = 0;   // chunks issued so far: stage gc & 1, phase gc >> 1 of that stage

  for (int64_t blk = first; blk * FTM < f.rows; blk += stride) {
    const int64_t p0 = blk * FTM;
    // 1. V for the block's rows, hi/lo TF32, into the resident K-major tiles.
    for (int ll = warp; ll < FTM; ll += FNT / 32) {
      const int64_t p = p0 + ll;
      const bool valid = p < f.rows;
      float* S = chain[warp];
      int Rs = 1;
      if (valid) {
        int64_t ii[kMaxModes];
        int64_t rem = p;
        for (int m = f.s - 1; m >= 0; --m) { ii[m] = rem % a.dims[m]; rem /= a.dims[m]; }
        Rs = warp_slice_product<float>(a, 0, f.s, ii, S, slice[warp], lane);
        __syncwarp();
      }
      for (int e = lane; e < Kc * FTK; e += 32) {
        float v = 0.f;
        if (valid && e < K) {
          const int b = e / Rlast, aa = e - b * Rlast;
          v = S[aa * Rs + b];
        }
        const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
        const int c = e / FTK, k = e - c * FTK;
        const uint32_t off = sw128_offset(ll, k);
        *reinterpret_cast<float*>(vt + c * 2 * FT_TILE + off) = hi;
        *reinterpret_cast<float*>(vt + c * 2 * FT_TILE + FT_TILE + off) = lo;
      }
      __syncwarp();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 2. Tiles of 128 columns.
    for (int64_t q0 = 0; q0 < f.cols; q0 += FTN) {
      for (int c = 0; c < Kc; ++c, ++gc) {
        const int s = static_cast<int>(gc & 1);
        unsigned char* st = stg + s * FT_STAGE;
        if (gc >= 2 && tid == 0) {   // the MMAs that last read this stage have finished
          if (!mbar_wait(smem_u32(&sh.mbar[s]), static_cast<uint32_t>(((gc - 2) >> 1) & 1)))
            sh.abort = 1;
        }
        __syncthreads();
        if (sh.abort) break;
        const int col = tid & (FTN - 1);
        const int64_t q = q0 + col;
#pragma unroll
        for (int r = 0; r < FTK / 2; ++r) {
          const int k = (tid >> 7) + 2 * r;
          const int e = c * FTK + k;
          const float w = (q < f.cols && e < K) ? WT[static_cast<int64_t>(e) * f.cols + q] : 0.f;
          const float hi = tf32_rna(w), lo = tf32_rna(w - hi);
          const uint32_t off = sw128_offset(col, k);
          *reinterpret_cast<float*>(st + off) = hi;
          *reinterpret_cast<float*>(st + FT_TILE + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_hi = smem_u32(vt + c * 2 * FT_TILE), a_lo = a_hi + FT_TILE;
          const uint32_t b_hi = smem_u32(st), b_lo = b_hi + FT_TILE;
#pragma unroll
          for (int ks = 0; ks < FTK / 8; ++ks) {
            const uint32_t koff = ks * 32;
            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
            mma_tf32(tmem, make_desc(a_hi + koff), make_desc(b_hi + koff), kIdesc, acc);
            mma_tf32(tmem, make_desc(a_hi + koff), make_desc(b_lo + koff), kIdesc, 1u);
            mma_tf32(tmem, make_desc(a_lo + koff), make_desc(b_hi + koff), kIdesc, 1u);
          }
          mma_commit(smem_u32(&sh.mbar[s]));
        }
      }
      if (sh.abort) break;
      // The tile's last commit covers all of its MMAs.
      if (tid == 0) {
        const long long gl = gc - 1;
        if (!mbar_wait(smem_u32(&sh.mbar[gl & 1]), static_cast<uint32_t>((gl >> 1) & 1)))
          sh.abort = 1;
      }
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (sh.abort) break;
      const int quarter = warp & 3, half = warp >> 2;
      const int64_t p = p0 + quarter * 32 + lane;
      float se_t = 0.f, sx_t = 0.f;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int col0 = half * 64 + cc * 32;
        float v[32];
        tmem_load32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) + col0, v);
        if (p < f.rows) {
          const float* xr = X + p * f.cols + q0 + col0;
          const int64_t left = f.cols - (q0 + col0);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            if (i < left) {
              const float x = xr[i];
              const float d = x - v[i];
              se_t += d * d;
              sx_t += x * x;
            }
          }
        }
      }
      se += static_cast<double>(se_t);
      sx += static_cast<double>(sx_t);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
    if (sh.abort) break;
  }
  // Wait (bounded) for every issued MMA before the tensor memory is freed.
  if (tid == 0 && gc > 0) {
    const long long gl = gc - 1;
    if (!mbar_wait(smem_u32(&sh.mbar[gl & 1]), static_cast<uint32_t>((gl >> 1) & 1)))
      sh.abort = 1;
    if (gl >= 1 &&
        !mbar_wait(smem_u32(&sh.mbar[(gl - 1) & 1]), static_cast<uint32_t>(((gl - 1) >> 1) & 1)))
      sh.abort = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem), "r"(kTmemCols) : "memory");
  if (tid == 0 && sh.abort) atomicOr(err, kErrTimeout);
}

}  // namespace trk
