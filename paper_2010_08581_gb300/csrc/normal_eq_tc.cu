// Row a5 on the 5th-generation tensor cores: C = A~^T [A~ | Y~] (M = A~^T A~ and B = A~^T Y~
// of the sampled LS, Alg. 2 LS step) with tcgen05.mma kind::tf32 and FP32 accumulation in
// tensor memory.
//
// Each FP32 operand x is split into TF32 parts hi = rna_tf32(x), lo = rna_tf32(x - hi), and
// every k-step issues hi*hi + hi*lo + lo*hi into the same accumulator, which recovers
// close to FP32 accuracy (Markidis et al., "NVIDIA Tensor Core Programmability,
// Performance & Precision", 2018; Ootomo & Yokota, 2022).
//
// One CTA = one 128 x BN output tile over one chunk of the J samples (split-K, partials
// reduced downstream in a fixed order). All 256 threads load the chunk from global memory
// (16-byte vectors along the feature / fibre index), split it and store it into K-major,
// 128-byte-swizzled shared-memory tiles; one elected thread issues the MMAs and commits
// them to an mbarrier per pipeline stage; TMEM is read back with tcgen05.ld. Every
// mbarrier wait is bounded: a wait of the main loop polls at most `wait_limit` times; on
// expiry the CTA records an error, stops issuing, waits (bounded by the default limit) for
// the MMAs it has committed, frees its TMEM and returns without writing its partials.
#include "common.cuh"
#include "tc_common.cuh"

namespace trk {
namespace {

constexpr int TM = 128;          // UMMA M
constexpr int TN = 128;          // UMMA N (output columns per CTA)
constexpr int TK = 32;           // samples per pipeline stage (one 128-byte swizzle row)
constexpr int NT = 256;
static_assert(TK == 32 && TM == 4 * (NT / 32) * 4,
              "operand loader: one sample per lane, 4 groups of 4 rows per warp");
constexpr int STAGES = 2;
constexpr int A_BYTES = TM * TK * 4;   // 16 KB
constexpr int B_BYTES = TN * TK * 4;   // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of both operands
constexpr uint32_t TMEM_COLS = TN;     // FP32 accumulator: 128 lanes x TN columns

using namespace tc;

constexpr uint32_t kIdesc = idesc_tf32(TM, TN);

__global__ void __launch_bounds__(NT, 1) k_normal_eq_tc(const float* __restrict__ A,
                                                        const float* __restrict__ Y, int64_t J,
                                                        int L, int64_t I, int64_t chunk,
                                                        float* __restrict__ partial,
                                                        unsigned* err, long long wait_limit,
                                                        const int64_t* __restrict__ jdev) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte alignment of the tiles (required by the 128-byte swizzle atoms)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t mbar[STAGES];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ldc = L + I;
  const int m0 = blockIdx.y * TM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * TN;
  const int64_t j0 = static_cast<int64_t>(blockIdx.z) * chunk;
  const int64_t Jr = jdev ? (*jdev < J ? *jdev : J) : J;
  const int64_t j1 = (j0 + chunk < Jr) ? j0 + chunk : Jr;
  const int nchunks = j1 > j0 ? static_cast<int>((j1 - j0 + TK - 1) / TK) : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(smem_u32(&mbar[s]), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = tmem_slot;

  // Loaders. Each thread holds TK/2 values of each operand per chunk: 4-wide groups g = u / 4
  // (u < TK/2) of 4 consecutive tile rows (features for A, output columns for B) at one
  // sample. With rows of A and Y that are multiples of 16 bytes long (and 16-byte aligned
  // bases) a group is one 16-byte load; otherwise four scalar loads with bounds.
  const bool vec = (L % 4) == 0 && (I % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(A) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(Y) % 16) == 0;
  // group q (0..3) of thread t: sample k = lane, tile rows 4 g .. 4 g + 3 with
  // g = warp + 8 q. Lanes cover consecutive samples, so the stores into the K-major swizzled
  // tile below hit 32 different banks (consecutive k of one row span the whole 128-byte line).
  auto load_chunk = [&](int c, float (&ra)[TK / 2], float (&rb)[TK / 2]) {
    const int64_t jb = j0 + static_cast<int64_t>(c) * TK;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = jb + lane;
      const int r4 = 4 * (warp + (NT / 32) * q);
      const int am = m0 + r4;
      const int64_t bn = n0 + r4;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (j < j1) {
        if (vec) {
          if (am < L) a = __ldg(reinterpret_cast<const float4*>(A + j * L + am));
          if (bn < L) b = __ldg(reinterpret_cast<const float4*>(A + j * L + bn));
          else if (bn < ldc) b = __ldg(reinterpret_cast<const float4*>(Y + j * I + (bn - L)));
        } else {
          float av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            av[i] = (am + i < L) ? __ldg(A + j * L + am + i) : 0.f;
            const int64_t c2 = bn + i;
            bv[i] = c2 < L ? __ldg(A + j * L + c2)
                           : (c2 < ldc ? __ldg(Y + j * I + (c2 - L)) : 0.f);
          }
          a = make_float4(av[0], av[1], av[2], av[3]);
          b = make_float4(bv[0], bv[1], bv[2], bv[3]);
        }
      }
      ra[4 * q] = a.x; ra[4 * q + 1] = a.y; ra[4 * q + 2] = a.z; ra[4 * q + 3] = a.w;
      rb[4 * q] = b.x; rb[4 * q + 1] = b.y; rb[4 * q + 2] = b.z; rb[4 * q + 3] = b.w;
    }
  };
  float ca[TK / 2], cb[TK / 2], na[TK / 2], nb[TK / 2];
  if (nchunks > 0) load_chunk(0, ca, cb);
  int issued = 0;

  for (int c = 0; c < nchunks; ++c) {
    const int s = c % STAGES;
    unsigned char* st = base + s * STAGE_BYTES;
    if (c + 1 < nchunks) load_chunk(c + 1, na, nb);   // in flight while this chunk is stored
    if (c >= STAGES) {   // wait until the MMAs that read this stage have finished
      const bool ok = mbar_wait(smem_u32(&mbar[s]), ((c / STAGES) - 1) & 1, wait_limit);
      if (!ok) atomicExch(&s_abort, 1);
    }
    __syncthreads();
    if (s_abort) break;
#pragma unroll
    for (int u = 0; u < TK / 2; ++u) {
      const int k = lane;
      const int row = 4 * (warp + (NT / 32) * (u / 4)) + (u % 4);
      const float a = ca[u], b = cb[u];
      const float ah = tf32_rna(a), bh = tf32_rna(b);
      const float al = tf32_rna(a - ah), bl = tf32_rna(b - bh);
      const uint32_t oa = sw128_offset(row, k);
      *reinterpret_cast<float*>(st + oa) = ah;
      *reinterpret_cast<float*>(st + A_BYTES + oa) = al;
      *reinterpret_cast<float*>(st + 2 * A_BYTES + oa) = bh;
      *reinterpret_cast<float*>(st + 2 * A_BYTES + B_BYTES + oa) = bl;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(st), a_lo = a_hi + A_BYTES;
      const uint32_t b_hi = a_hi + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
#pragma unroll
      for (int ks = 0; ks < TK / 8; ++ks) {
        const uint32_t koff = ks * 32;   // 8 TF32 = 32 bytes along K inside the swizzle row
        const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem_d, make_desc(a_hi + koff), make_desc(b_hi + koff), kIdesc, acc0);
        mma_tf32(tmem_d, make_desc(a_hi + koff), make_desc(b_lo + koff), kIdesc, 1u);
        mma_tf32(tmem_d, make_desc(a_lo + koff), make_desc(b_hi + koff), kIdesc, 1u);
      }
      mma_commit(smem_u32(&mbar[s]));
    }
    issued = c + 1;
#pragma unroll
    for (int r = 0; r < TK / 2; ++r) { ca[r] = na[r]; cb[r] = nb[r]; }
  }
  __syncthreads();
  const int aborted = s_abort;
  // `issued` counts the chunks whose MMAs were committed: all of them, or, after an expired
  // wait at chunk c, chunks 0 .. c-1.
  // Wait for the last commit of each stage that was used (bounded by the default limit,
  // so that no MMA is in flight when TMEM is freed).
  bool ok = true;
  if (issued > 0) {
    const int last = issued - 1;
    ok = mbar_wait(smem_u32(&mbar[last % STAGES]), (last / STAGES) & 1);
    if (issued > 1) {
      const int prev = issued - 2;
      ok = mbar_wait(smem_u32(&mbar[prev % STAGES]), (prev / STAGES) & 1) && ok;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) atomicExch(&s_abort, 1);
  __syncthreads();
  const bool failed = aborted || s_abort != 0;     // the same for every thread
  if (failed) {
    if (tid == 0) atomicOr(err, kErrTimeout);
  } else if (issued == 0) {
    // no rows in this chunk (beyond the device-side row count): zero partials
    for (int e = tid; e < TM * TN; e += NT) {
      const int m = m0 + e / TN;
      const int64_t col = n0 + e % TN;
      if (m < L && col < ldc)
        partial[(static_cast<int64_t>(blockIdx.z) * L + m) * ldc + col] = 0.0f;
    }
  } else {
    // Epilogue through shared memory (every MMA has completed, so the stage buffers are
    // free): warp w moves TMEM lanes 32*(w%4).. (tile rows) of column half w/4 into a
    // [TM][TN + 1] tile (odd stride: no bank conflicts), then the warps write whole rows,
    // 32 consecutive columns per store instruction.
    float* tile = reinterpret_cast<float*>(base);
    const int quad = warp & 3, half = warp >> 2;
    const int rl = quad * 32 + lane;
#pragma unroll
    for (int cc = 0; cc < TN / 64; ++cc) {
      const int col = half * (TN / 2) + cc * 32;
      float v[32];
      tmem_load32(tmem_d + (static_cast<uint32_t>(quad * 32) << 16) + col, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) tile[rl * (TN + 1) + col + i] = v[i];
    }
    __syncthreads();
    for (int r = warp; r < TM; r += NT / 32) {
      const int m = m0 + r;
      if (m >= L) break;
      float* out = partial + (static_cast<int64_t>(blockIdx.z) * L + m) * ldc + n0;
#pragma unroll
      for (int q = 0; q < TN / 32; ++q) {
        const int c = lane + 32 * q;
        if (n0 + c < ldc) out[c] = tile[r * (TN + 1) + c];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tmem_d), "r"(TMEM_COLS) : "memory");
}

void plan_tc(int64_t J, int L, int64_t I, int* splits, int64_t* chunk) {
  const int64_t tiles = ((L + TM - 1) / TM) * ((L + I + TN - 1) / TN);
  int64_t s = (sm_count() + tiles - 1) / tiles;
  const int64_t maxs = (J + 4 * TK - 1) / (4 * TK);   // at least 4 stages per CTA
  if (s > maxs) s = maxs;
  if (s < 1) s = 1;
  int64_t c = (J + s - 1) / s;
  c = (c + TK - 1) / TK * TK;
  s = (J + c - 1) / c;
  *splits = static_cast<int>(s);
  *chunk = c;
}

}  // namespace

size_t normal_eq_tc_workspace(int64_t J, int L, int64_t I, int* splits) {
  int64_t chunk;
  plan_tc(J, L, I, splits, &chunk);
  return static_cast<size_t>(*splits) * L * (L + I) * sizeof(float);
}

cudaError_t launch_normal_eq_tc(const float* A, const float* Y, int64_t J, int L, int64_t I,
                                float* partial, int splits, unsigned* err, cudaStream_t st,
                                long long wait_limit, const int64_t* jdev) {
  int s;
  int64_t chunk;
  plan_tc(J, L, I, &s, &chunk);
  if (s != splits) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned>((L + I + TN - 1) / TN), (L + TM - 1) / TM, s);
  const size_t dyn = STAGES * STAGE_BYTES + 1024;
  k_normal_eq_tc<<<grid, NT, dyn, st>>>(A, Y, J, L, I, chunk, partial, err,
                                        wait_limit < 0 ? kTcSpinLimit : wait_limit, jdev);
  return cudaGetLastError();
}

cudaError_t normal_eq_tc_attributes() {
  return cudaFuncSetAttribute(k_normal_eq_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              STAGES * STAGE_BYTES + 1024);
}

}  // namespace trk
