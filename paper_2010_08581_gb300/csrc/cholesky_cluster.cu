// FP64 Cholesky factorisation G = L L^T (rows a1 and a6: the leverage scores of Def. 4 and
// the LS step of Alg. 2) on a thread-block cluster of CC CTAs, for n <= kClusterMaxN: the
// single-problem drivers' factorisations, whose one-CTA form is bounded by one SM's FP64
// pipe.
//
// Column j is owned by CTA j % CC; CTA c keeps its columns in registers, thread i holding
// row i. Right-looking with one column of look-ahead: when column k is final, its owner
// writes it into its own column buffer k and sends the buffer to every other CTA that still
// needs it with one bulk copy (distributed shared memory) that completes the transaction
// bytes of that CTA's mbarrier k (armed once with the copy's size). Every CTA waits for
// column k; the owner of column k+1 applies it to that column first, finalises and sends
// column k+1; then every CTA applies column k to the rest of its columns. Each buffer and
// mbarrier is written once, so there is no reuse to order. Per element the updates, the
// pivot test and the scaling are the same operations in the same order as the one-CTA
// kernel (cholesky_body.cuh), so the factors are identical.
//
// mode 0 (solve): a pivot <= tol_scale * max diag stops the factorisation (*info = column
// + 1, singular bit); the stop travels with the column to every CTA. mode 1 (leverage): such
// a column becomes zero and keep = 0. Every wait is bounded; on expiry the CTA records the
// timeout bit and leaves the loop. All CTAs meet at a final cluster barrier so that no CTA
// exits while another may still write into its shared memory.
#include "common.cuh"

namespace trk {
namespace {

constexpr int CC = 8;                           // CTAs per cluster
constexpr int CCT = 256;                        // threads per CTA: thread i owns row i
constexpr int kClusterMaxN = 144;               // n x (n+1) FP64 buffers fit in shared memory
constexpr int kMaxLoc = (kClusterMaxN + CC - 1) / CC;
constexpr long long kClusterSpin = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// Bulk copy of `bytes` (a multiple of 16) from this CTA's shared memory to another CTA's
// shared memory in the cluster, completing that many transaction bytes of its mbarrier.
__device__ __forceinline__ void copy_to_rank(uint32_t dst, uint32_t src, uint32_t bytes,
                                             uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :: "r"(dst), "r"(src), "r"(bytes), "r"(bar) : "memory");
}

// Column j is sent from row j & ~1 to the end of its buffer (16-byte aligned and sized).
__device__ __forceinline__ int col_send_first(int j) { return j & ~1; }

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Spin on the column's barrier without suspending (test_wait), bounded.
__device__ __forceinline__ bool wait_column(uint32_t bar) {
  for (long long it = 0; it < kClusterSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar) : "memory");
    if (done) return true;
  }
  return false;
}

// Last column owned by CTA r (-1 if none): CTA r needs column k iff k < last_owned(r, n).
__device__ __forceinline__ int last_owned(int r, int n) {
  return r < n ? r + CC * ((n - r + CC - 1) / CC - 1) : -1;
}

__global__ void __cluster_dims__(CC, 1, 1) __launch_bounds__(CCT)
    k_cholesky_cluster(const double* __restrict__ G, int n, int mode, double tol_scale,
                       double* Lrow, double* Lcol, double* invdiag, int* keep_out, int* info,
                       unsigned* err, double* img64, float* img32, float* gimg32) {
  // Column buffers [n][cs]: rows 0..n-1 of column k, its stop flag at n; cs = n + 1 rounded up
  // to an even count so that every buffer starts on a 16-byte boundary.
  extern __shared__ __align__(16) double cbuf[];
  const int cs = (n + 2) & ~1;
  uint64_t* bars = reinterpret_cast<uint64_t*>(cbuf + n * cs);
  __shared__ double s_piv, s_tol;
  __shared__ int s_keep[kMaxLoc];
  __shared__ double s_red[CCT / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = static_cast<int>(cluster_rank());
  const int np = n + 1;                        // row stride of the padded factor images
  const int nloc = c < n ? (n - c + CC - 1) / CC : 0;
  const bool row = tid < n;

  // Owned columns j = c + CC * jl of row tid (lower triangle), and the FP32 image of G.
  double a[kMaxLoc];
#pragma unroll
  for (int jl = 0; jl < kMaxLoc; ++jl) {
    const int j = c + CC * jl;
    a[jl] = 0.0;
    if (jl < nloc && row && tid >= j) {
      const double g = G[static_cast<int64_t>(j) * n + tid];
      a[jl] = g;
      if (gimg32) {
        gimg32[j * np + tid] = static_cast<float>(g);
        gimg32[tid * np + j] = static_cast<float>(g);
      }
    }
  }
  // Pivot tolerance from the largest diagonal entry (same in every CTA).
  double md = row ? G[static_cast<int64_t>(tid) * n + tid] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
  if (lane == 0) s_red[warp] = md;
  // Column k is sent only to the CTAs that still need it (k < their last column). Their
  // barrier k expects the bytes of the column's bulk copy (rows k & ~1 .. the flag and pad),
  // and each of them waits for it before the final cluster barrier, so no copy is in flight
  // when a CTA leaves.
  const int jmine = last_owned(c, n);
  for (int k = tid; k < n; k += CCT) {
    const uint32_t b = smem_u32(&bars[k]);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b) : "memory");
    if (k % CC != c && k < jmine)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(b), "r"((cs - col_send_first(k)) * 8) : "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < CCT / 32; ++w) m = fmax(m, s_red[w]);
    s_tol = tol_scale * m;
  }
  cluster_sync_all();   // every CTA's barriers exist before any remote arrive
  const double tol = s_tol;

  int stop = 0;          // 1-based column of a failed pivot (mode 0), -1 on a timeout
  // Finalise owned column j (all updates applied): pivot, scale, send to every CTA.
  auto finalize = [&](int j) {
    const int jl = j / CC;
    if (tid == j) {
#pragma unroll
      for (int q = 0; q < kMaxLoc; ++q)
        if (q == jl) s_piv = a[q];
    }
    __syncthreads();
    const double d = s_piv;
    const bool ok = d > tol;                  // false for NaN and non-positive pivots
    const double inv = ok ? rsqrt(d) : 0.0;
    double* col = cbuf + j * cs;
    if (row && tid >= j) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < kMaxLoc; ++q)
        if (q == jl) {
          v = ok ? ((tid == j) ? d * inv : a[q] * inv) : 0.0;
          a[q] = v;
        }
      col[tid] = v;
    }
    if (tid == 0) {
      col[n] = (!ok && mode == 0) ? static_cast<double>(j + 1) : 0.0;
      s_keep[jl] = ok ? 1 : 0;
    }
    __syncthreads();
    // One bulk copy per CTA that needs the column, issued by thread r.
    if (tid < CC && tid != c && j < last_owned(tid, n)) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int f0 = col_send_first(j);
      const uint32_t src = smem_u32(col + f0);
      copy_to_rank(map_rank(src, tid), src, static_cast<uint32_t>((cs - f0) * 8),
                   map_rank(smem_u32(&bars[j]), tid));
    }
  };

  const int jlast = jmine;
  if (c == 0) {
    finalize(0);
    if (cbuf[n] != 0.0) stop = static_cast<int>(cbuf[n]);
  }
  for (int k = 0; stop == 0 && k < jlast; ++k) {
    if (k % CC != c) {
      // one thread spins (acquire at cluster scope); the CTA barrier then orders the other
      // threads' reads after it, and the CTA leaves together if the wait expired
      const bool ok = (tid == 0) ? wait_column(smem_u32(&bars[k])) : true;
      if (__syncthreads_or(ok ? 0 : 1)) {
        if (tid == 0) atomicOr(err, kErrTimeout);
        stop = -1;
        break;
      }
    }
    const double* col = cbuf + k * cs;
    const double flag = col[n];
    if (flag != 0.0) {
      stop = static_cast<int>(flag);
      break;
    }
    const double bi = (row && tid > k) ? col[tid] : 0.0;
    const int k1 = k + 1;
    const bool own_next = (k1 % CC) == c;
    if (own_next) {
      const int jl1 = k1 / CC;
      const double l1 = col[k1];
      if (row && tid >= k1) {
#pragma unroll
        for (int q = 0; q < kMaxLoc; ++q)
          if (q == jl1) a[q] = fma(-bi, l1, a[q]);
      }
      finalize(k1);
      if (cbuf[k1 * cs + n] != 0.0) {   // this CTA's own pivot failed (mode 0)
        stop = static_cast<int>(cbuf[k1 * cs + n]);
        break;
      }
    }
    if (row) {
#pragma unroll
      for (int q = 0; q < kMaxLoc; ++q) {
        const int j = c + CC * q;
        if (q < nloc && j > k && j != k1 && tid >= j) a[q] = fma(-bi, col[j], a[q]);
      }
    }
  }

  // The owner of column n-1 has seen every column's flag: it reports the status.
  if (c == (n - 1) % CC && tid == 0) {
    *info = stop > 0 ? stop : 0;
    if (stop > 0) atomicOr(err, kErrSingular);
  }
  if (stop == 0) {
#pragma unroll
    for (int q = 0; q < kMaxLoc; ++q) {
      const int j = c + CC * q;
      if (q >= nloc || !row) continue;
      const double v = tid >= j ? a[q] : 0.0;
      Lrow[static_cast<int64_t>(tid) * n + j] = v;
      Lcol[static_cast<int64_t>(j) * n + tid] = v;
      if (img64) img64[j * np + tid] = v;
      if (img32) img32[j * np + tid] = static_cast<float>(v);
      if (tid == j) {
        keep_out[j] = s_keep[q];
        invdiag[j] = s_keep[q] ? 1.0 / v : 0.0;
      }
    }
  }
  cluster_sync_all();   // no CTA leaves while another may still write into its buffers
}

}  // namespace

bool cholesky_cluster_fits(int n) { return n >= 1 && n <= kClusterMaxN; }

cudaError_t launch_cholesky_cluster(const double* G, int n, int mode, double tol_scale,
                                    double* Lrow, double* Lcol, double* invdiag, int* keep,
                                    int* info, unsigned* err, cudaStream_t st, double* img64,
                                    float* img32, float* gimg32) {
  const size_t dyn = static_cast<size_t>(n) * ((n + 2) & ~1) * sizeof(double) + n * sizeof(uint64_t);
  k_cholesky_cluster<<<CC, CCT, dyn, st>>>(G, n, mode, tol_scale, Lrow, Lcol, invdiag, keep,
                                           info, err, img64, img32, gimg32);
  return cudaGetLastError();
}

cudaError_t cholesky_cluster_attributes() {
  const int dyn = kClusterMaxN * ((kClusterMaxN + 2) & ~1) * 8 + kClusterMaxN * 8;
  return cudaFuncSetAttribute(k_cholesky_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              dyn);
}

}  // namespace trk
