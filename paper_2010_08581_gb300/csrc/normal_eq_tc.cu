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
// (coalesced along the feature / fibre index), split it and store it into K-major,
// 128-byte-swizzled shared-memory tiles; one elected thread issues the MMAs and commits
// them to an mbarrier per pipeline stage; TMEM is read back with tcgen05.ld. Every
// mbarrier wait is bounded: on expiry the CTA records an error, waits (bounded) for its
// outstanding MMAs, frees its TMEM and returns.
#include "common.cuh"
#include "tc_common.cuh"

namespace trk {
namespace {

constexpr int TM = 128;          // UMMA M
constexpr int TN = 128;          // UMMA N (output columns per CTA)
constexpr int TK = 32;           // samples per pipeline stage (one 128-byte swizzle row)
constexpr int NT = 256;
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
                                                        unsigned* err) {
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
  const int64_t j1 = (j0 + chunk < J) ? j0 + chunk : J;
  const int nchunks = static_cast<int>((j1 - j0 + TK - 1) / TK);

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

  // Element loaders: thread t covers row (t % 128) of the tile and samples k = t/128 + 2r.
  const int row = tid & 127;
  const int k_first = tid >> 7;
  const int am = m0 + row;                    // feature index of the A operand
  const int64_t bn = n0 + row;                // output column of the B operand
  // Raw FP32 values of one chunk for this thread: samples k_first + 2r, r < TK/2.
  auto load_chunk = [&](int c, float (&ra)[TK / 2], float (&rb)[TK / 2]) {
    const int64_t jb = j0 + static_cast<int64_t>(c) * TK;
#pragma unroll
    for (int r = 0; r < TK / 2; ++r) {
      const int64_t j = jb + k_first + 2 * r;
      float a = 0.f, b = 0.f;
      if (j < j1) {
        if (am < L) a = __ldg(A + j * L + am);
        if (bn < L) b = __ldg(A + j * L + bn);
        else if (bn < ldc) b = __ldg(Y + j * I + (bn - L));
      }
      ra[r] = a;
      rb[r] = b;
    }
  };
  float ca[TK / 2], cb[TK / 2], na[TK / 2], nb[TK / 2];
  if (nchunks > 0) load_chunk(0, ca, cb);

  for (int c = 0; c < nchunks; ++c) {
    const int s = c % STAGES;
    unsigned char* st = base + s * STAGE_BYTES;
    if (c + 1 < nchunks) load_chunk(c + 1, na, nb);   // in flight while this chunk is stored
    if (c >= STAGES) {   // wait until the MMAs that read this stage have finished
      const bool ok = mbar_wait(smem_u32(&mbar[s]), ((c / STAGES) - 1) & 1);
      if (!ok) atomicExch(&s_abort, 1);
    }
    __syncthreads();
    if (s_abort) break;
#pragma unroll
    for (int r = 0; r < TK / 2; ++r) {
      const int k = k_first + 2 * r;
      const float a = ca[r], b = cb[r];
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
#pragma unroll
    for (int r = 0; r < TK / 2; ++r) { ca[r] = na[r]; cb[r] = nb[r]; }
  }
  __syncthreads();
  const int aborted = s_abort;
  // Wait for the last commit of each stage that was used (bounded).
  bool ok = true;
  if (nchunks > 0) {
    const int last = nchunks - 1;
    ok = mbar_wait(smem_u32(&mbar[last % STAGES]), (last / STAGES) & 1);
    if (nchunks > 1) {
      const int prev = nchunks - 2;
      ok = mbar_wait(smem_u32(&mbar[prev % STAGES]), (prev / STAGES) & 1) && ok;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok || aborted) {
    if (tid == 0) atomicOr(err, kErrTimeout);
  } else if (nchunks > 0) {
    // Epilogue: warp w reads TMEM lanes 32*(w%4).. (rows) and column half w/4.
    const int quad = warp & 3, half = warp >> 2;
    const int m = m0 + quad * 32 + lane;
#pragma unroll
    for (int cc = 0; cc < TN / 64; ++cc) {
      const int col = half * (TN / 2) + cc * 32;
      float v[32];
      tmem_load32(tmem_d + (static_cast<uint32_t>(quad * 32) << 16) + col, v);
      if (m < L) {
        float* out = partial + (static_cast<int64_t>(blockIdx.z) * L + m) * ldc + n0 + col;
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (n0 + col + i < ldc) out[i] = v[i];
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
                                float* partial, int splits, unsigned* err, cudaStream_t st) {
  int s;
  int64_t chunk;
  plan_tc(J, L, I, &s, &chunk);
  if (s != splits) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned>((L + I + TN - 1) / TN), (L + TM - 1) / TM, s);
  const size_t dyn = STAGES * STAGE_BYTES + 1024;
  k_normal_eq_tc<<<grid, NT, dyn, st>>>(A, Y, J, L, I, chunk, partial, err);
  return cudaGetLastError();
}

cudaError_t normal_eq_tc_attributes() {
  return cudaFuncSetAttribute(k_normal_eq_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              STAGES * STAGE_BYTES + 1024);
}

}  // namespace trk
