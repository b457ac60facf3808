// The relative-error contraction of fit_body.cuh (the error ||TR - X|| / ||X|| of Sec. 5
// and the stop rule of Sec. 4.1) on the 5th-generation tensor cores, for X in FP32 and
// contraction length K <= 128.
//
// The right factors W are formed once per evaluation (fit_right_tc_warp) already split
// into TF32 parts hi = rna(w), lo = rna(w - hi) and laid out as the MMA's K-major,
// 128-byte-swizzled operand tiles: [column tile][K chunk][hi 16 KB | lo 16 KB]. Per block of
// 128 rows the CTA forms V (the left slice products, build_left), splits it the same way and
// keeps it in shared memory for the whole block. For every tile of 128 columns one elected
// thread streams the K chunks (32 wide) of W through two shared-memory stages with one bulk
// copy each (transaction-byte mbarriers, one chunk ahead) and issues hi*hi + hi*lo + lo*hi
// per 8-wide k-step into one FP32 accumulator in tensor memory (about FP32 accuracy),
// committing each chunk to the stage's second mbarrier. The epilogue reads TR(p, q) back from tensor memory (warp w: rows 32 (w % 4)..,
// columns 64 (w / 4)..), forms (X - TR)^2 and X^2 in FP32 per tile and adds them to FP64
// per-thread totals. Every mbarrier wait is bounded: on expiry the CTA records the timeout
// bit, waits (bounded) for its issued MMAs, frees its tensor memory and stops.
#pragma once

#include "fit_body.cuh"
#include "tc_common.cuh"

namespace trk {

constexpr int kFitTcMaxK = 256;
constexpr int FT_KG = 4;                          // K chunks resident in shared memory (128)
constexpr int FT_TG = 4;                          // column tiles accumulated at once (TMEM)
constexpr int FTM = 128;                          // rows per block (MMA M)
constexpr int FTN = 128;                          // columns per tile (MMA N)
constexpr int FTK = 32;                           // K per chunk (one 128-byte swizzle row)
constexpr int FT_TILE = FTM * FTK * 4;            // 16 KB: hi or lo of one operand chunk
constexpr int FT_VBYTES = 2 * FT_KG * FT_TILE;   // V hi/lo of one K group
constexpr int FT_STAGE = 2 * FT_TILE;             // W chunk hi + lo
constexpr size_t kFitTcSmem = FT_VBYTES + 2 * FT_STAGE + 1024;

// Bytes of the swizzled right factors for a split: column tiles x K chunks x (hi + lo).
__host__ __device__ inline size_t fit_tc_right_bytes(const FitSplit& f) {
  const int64_t tiles = (f.cols + FTN - 1) / FTN;
  const int Kc = (f.K + FTK - 1) / FTK;
  return static_cast<size_t>(tiles) * Kc * FT_STAGE;
}

// The tensor-core contraction serves FP32 X with K <= 128; the rest uses fit_blocks.
__host__ __device__ inline bool fit_use_tc(const FitSplit& f, bool xf64) {
  return !xf64 && f.K <= kFitTcMaxK;
}

__host__ __device__ inline int64_t fit_row_blocks(const FitSplit& f, bool xf64) {
  const int64_t rb = fit_use_tc(f, xf64) ? FTM : (xf64 ? FitTile<double>::FL : FitTile<float>::FL);
  return (f.rows + rb - 1) / rb;
}

struct FitTcShared {
  uint64_t full[2];     // a stage's bulk copy has landed (transaction bytes)
  uint64_t empty[2];    // the MMAs that read a stage have finished (tcgen05.commit)
  uint32_t tmem_slot;
  int abort;
};

// Column q (< column tiles * 128) of the swizzled right factors, one warp; q >= cols and
// entries e >= K are zero. S and G are per-warp scratch of kMaxL elements.
__device__ inline void fit_right_tc_warp(const FitArgs& a, const FitSplit& f, int64_t q,
                                         unsigned char* __restrict__ WS, float* S, float* G,
                                         int lane) {
  using namespace tc;
  const int N = a.N;
  const int Kc = (f.K + FTK - 1) / FTK;
  const bool valid = q < f.cols;
  if (valid) {
    int64_t ii[kMaxModes];
    int64_t rem = q;
    for (int m = N - 1; m >= f.s; --m) { ii[m] = rem % a.dims[m]; rem /= a.dims[m]; }
    warp_slice_product<float>(a, f.s, N, ii, S, G, lane);
    __syncwarp();
  }
  const int64_t t = q / FTN;
  const int col = static_cast<int>(q - t * FTN);
  for (int e = lane; e < Kc * FTK; e += 32) {
    const float w = (valid && e < f.K) ? S[e] : 0.f;
    const float hi = tf32_rna(w), lo = tf32_rna(w - hi);
    const int c = e / FTK, k = e - c * FTK;
    unsigned char* tile = WS + (static_cast<size_t>(t) * Kc + c) * FT_STAGE;
    const uint32_t off = sw128_offset(col, k);
    *reinterpret_cast<float*>(tile + off) = hi;
    *reinterpret_cast<float*>(tile + FT_TILE + off) = lo;
  }
  __syncwarp();
}

// Accumulates (se, sx) over the row blocks first, first + stride, ... All threads of the CTA
// call it; `dyn` holds kFitTcSmem bytes of dynamic shared memory.
__device__ inline void fit_tc_blocks(const FitArgs& a, const FitSplit& f,
                                     const float* __restrict__ X,
                                     const unsigned char* __restrict__ WS,
                                     int64_t first, int64_t stride, unsigned char* dyn,
                                     float (*chain)[kMaxL], float (*slice)[kMaxL],
                                     FitTcShared& sh, unsigned* err, double& se, double& sx) {
  using namespace tc;
  constexpr uint32_t kIdesc = idesc_tf32(FTM, FTN);
  constexpr uint32_t kTmemCols = FT_TG * FTN;   // 512: one accumulator per tile of a group
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
  unsigned char* vt = base;                 // chunk c: hi at c * 2 * FT_TILE, lo after it
  unsigned char* stg = base + FT_VBYTES;    // stage s: hi at s * FT_STAGE, lo after it
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = f.K, Kc = (K + FTK - 1) / FTK;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&sh.tmem_slot)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&sh.full[q]), 1);
      mbar_init(smem_u32(&sh.empty[q]), 1);
    }
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem_slot;
  // Per row block the chunks run in the order: column groups of up to FT_TG tiles, then K
  // groups of up to FT_KG chunks, then the group's tiles, then the K group's chunks. Chunk
  // g of this CTA uses stage g & 1, phase g >> 1 of its barriers.
  const int64_t tiles = (f.cols + FTN - 1) / FTN;
  const int nkg = (Kc + FT_KG - 1) / FT_KG;
  const long long per_block = tiles * Kc;
  const int64_t my_blocks = (first * FTM < f.rows)
                                ? ((f.rows + FTM - 1) / FTM - first + stride - 1) / stride : 0;
  const long long total = my_blocks * per_block;
  // (tile, chunk) of the r-th chunk of a row block
  auto chunk_of = [&](long long r, int64_t* t, int* c) {
    const long long gi = r / (static_cast<long long>(FT_TG) * Kc);
    long long r1 = r - gi * FT_TG * Kc;
    const int gt = static_cast<int>(tiles - gi * FT_TG < FT_TG ? tiles - gi * FT_TG : FT_TG);
    const int kg = static_cast<int>(r1 / (static_cast<long long>(gt) * FT_KG));
    r1 -= static_cast<long long>(kg) * gt * FT_KG;
    const int kc = Kc - kg * FT_KG < FT_KG ? Kc - kg * FT_KG : FT_KG;
    *t = gi * FT_TG + r1 / kc;
    *c = kg * FT_KG + static_cast<int>(r1 % kc);
  };
  long long g = 0;          // next chunk to consume (thread 0)
  long long issued = -1;    // last chunk whose copy was issued (thread 0)
  auto issue = [&](long long h) {   // thread 0: copy chunk h into stage h & 1
    const int s = static_cast<int>(h & 1);
    if (h >= 2 && !mbar_wait(smem_u32(&sh.empty[s]), static_cast<uint32_t>(((h - 2) >> 1) & 1))) {
      sh.abort = 1;
      return;
    }
    int64_t t;
    int c;
    chunk_of(h % per_block, &t, &c);
    const unsigned char* src = WS + (static_cast<size_t>(t) * Kc + c) * FT_STAGE;
    const uint32_t full = smem_u32(&sh.full[s]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(full), "r"(static_cast<uint32_t>(FT_STAGE)) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_u32(stg + s * FT_STAGE)), "l"(src), "r"(static_cast<uint32_t>(FT_STAGE)),
           "r"(full) : "memory");
    issued = h;
  };
  if (tid == 0 && total > 0) issue(0);

  for (int64_t blk = first; blk * FTM < f.rows; blk += stride) {
    const int64_t p0 = blk * FTM;
    for (int64_t gi = 0; gi * FT_TG < tiles; ++gi) {
      const int gt = static_cast<int>(tiles - gi * FT_TG < FT_TG ? tiles - gi * FT_TG : FT_TG);
      for (int kg = 0; kg < nkg; ++kg) {
        const int kc = Kc - kg * FT_KG < FT_KG ? Kc - kg * FT_KG : FT_KG;
        // 1. V for the block's rows and this K group, hi/lo TF32, into the resident
        // K-major tiles (entries K .. of the last group are zero). With one K group V is
        // formed once per row block.
        if (nkg > 1 || gi == 0) {
          const int e0 = kg * FT_KG * FTK, e1 = e0 + kc * FTK;
          auto put = [&](int ll, int e, float v) {
            const float hi = tf32_rna(v), lo = tf32_rna(v - hi);
            const int c = (e - e0) / FTK, k = (e - e0) - c * FTK;
            const uint32_t off = sw128_offset(ll, k);
            *reinterpret_cast<float*>(vt + c * 2 * FT_TILE + off) = hi;
            *reinterpret_cast<float*>(vt + c * 2 * FT_TILE + FT_TILE + off) = lo;
          };
          const int kpad0 = K > e0 ? K : e0;
          const int pad = e1 - kpad0;
          for (int it = tid; it < FTM * pad; it += FNT) put(it / pad, kpad0 + it % pad, 0.f);
          build_left<float>(a, f, p0, FTM, e0, e1, chain, slice, put);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncthreads();
        }
        // 2. The group's tiles over this K group's chunks, one elected thread.
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int j = 0; j < gt && !sh.abort; ++j) {
            for (int c = 0; c < kc && !sh.abort; ++c, ++g) {
              if (g + 1 < total) issue(g + 1);   // one chunk ahead
              if (sh.abort) break;
              const int s = static_cast<int>(g & 1);
              if (!mbar_wait(smem_u32(&sh.full[s]), static_cast<uint32_t>((g >> 1) & 1))) {
                sh.abort = 1;
                break;
              }
              const uint32_t a_hi = smem_u32(vt + c * 2 * FT_TILE), a_lo = a_hi + FT_TILE;
              const uint32_t b_hi = smem_u32(stg + s * FT_STAGE), b_lo = b_hi + FT_TILE;
              const uint32_t acc_t = tmem + static_cast<uint32_t>(j * FTN);
#pragma unroll
              for (int ks = 0; ks < FTK / 8; ++ks) {
                const uint32_t koff = ks * 32;
                const uint32_t acc = (kg > 0 || c > 0 || ks > 0) ? 1u : 0u;
                mma_tf32(acc_t, make_desc(a_hi + koff), make_desc(b_hi + koff), kIdesc, acc);
                mma_tf32(acc_t, make_desc(a_hi + koff), make_desc(b_lo + koff), kIdesc, 1u);
                mma_tf32(acc_t, make_desc(a_lo + koff), make_desc(b_hi + koff), kIdesc, 1u);
              }
              mma_commit(smem_u32(&sh.empty[s]));
            }
          }
          // The K group's last commit covers all of its MMAs (V may then be replaced).
          if (!sh.abort) {
            const long long gl = g - 1;
            if (!mbar_wait(smem_u32(&sh.empty[gl & 1]), static_cast<uint32_t>((gl >> 1) & 1)))
              sh.abort = 1;
          }
        }
        __syncthreads();
        if (sh.abort) break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (sh.abort) break;
      // 3. Epilogue of the group's tiles: warp w reads rows 32 (w % 4).., columns 64 (w / 4)..
      const int quarter = warp & 3, half = warp >> 2;
      const int64_t p = p0 + quarter * 32 + lane;
      float se_t = 0.f, sx_t = 0.f;
      for (int j = 0; j < gt; ++j) {
        const int64_t q0 = (gi * FT_TG + j) * FTN;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int col0 = half * 64 + cc * 32;
          float v[32];
          tmem_load32(tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                          static_cast<uint32_t>(j * FTN + col0), v);
          if (p < f.rows) {
            const float* xr = X + p * f.cols + q0 + col0;
            const int64_t left = f.cols - (q0 + col0);
            if (left >= 32 && (reinterpret_cast<uintptr_t>(xr) & 15) == 0) {
              float4 xv[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) xv[u] = __ldg(reinterpret_cast<const float4*>(xr) + u);
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const float xs[4] = {xv[u].x, xv[u].y, xv[u].z, xv[u].w};
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                  const float d = xs[jj] - v[4 * u + jj];
                  se_t += d * d;
                  sx_t += xs[jj] * xs[jj];
                }
              }
            } else {
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
        }
      }
      se += static_cast<double>(se_t);
      sx += static_cast<double>(sx_t);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
    if (sh.abort) break;
  }
  // Wait (bounded) for every issued MMA and bulk copy before the tensor memory is freed
  // and the CTA leaves.
  if (tid == 0) {
    if (g > 0 && !mbar_wait(smem_u32(&sh.empty[(g - 1) & 1]),
                            static_cast<uint32_t>(((g - 1) >> 1) & 1)))
      sh.abort = 1;
    if (issued >= g && !mbar_wait(smem_u32(&sh.full[issued & 1]),
                                  static_cast<uint32_t>((issued >> 1) & 1)))
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
