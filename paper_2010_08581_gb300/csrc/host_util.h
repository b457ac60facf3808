// Host-side helpers shared by the C ABI (api.cu) and the serving layer (server.cu): device
// guard, workspace carving, and the launch sequence of one batched step.
#pragma once

#include <cstdint>

#include "batched.cuh"

namespace trk {

// Makes `dev` current for the lifetime of the guard and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Bump allocator over a device region, 256-byte aligned. With base == nullptr it only
// measures.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b, size_t start = 0) : base(b), off(start) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

inline void row_major_strides(int N, const int64_t* dims, int64_t* stride) {
  int64_t s = 1;
  for (int k = N - 1; k >= 0; --k) { stride[k] = s; s *= dims[k]; }
}

inline size_t img_bytes(int n, bool f32) { return n > 0 ? trsm_image_bytes(n, f32) : 0; }

// Per-problem extents that size the batched scratch: sum and max of I_k, max L_k, and the
// Gram sizes of the two leverage passes (pass 2 only for wide modes, I_k < L_k).
struct BSizes {
  int64_t Isum = 0, Imax = 0;
  int Lmax = 0, n1 = 0, n2 = 0;
};

inline BSizes bsizes(int N, const int64_t* dims, const int* ranks) {
  BSizes z;
  for (int k = 0; k < N; ++k) {
    const int64_t I = dims[k];
    const int L = ranks[(k - 1 + N) % N] * ranks[k];
    z.Isum += I;
    z.Imax = I > z.Imax ? I : z.Imax;
    z.Lmax = L > z.Lmax ? L : z.Lmax;
    const int g1 = I >= L ? L : static_cast<int>(I);
    z.n1 = g1 > z.n1 ? g1 : z.n1;
    if (I < L) z.n2 = static_cast<int>(I) > z.n2 ? static_cast<int>(I) : z.n2;
  }
  return z;
}

// Carves one problem's distributions and per-update scratch (base == nullptr: measure only).
inline void carve_instance(Carver& c, int N, const int64_t* dims, const int* ranks, int64_t J,
                           bool f64, BInst& d) {
  const BSizes z = bsizes(N, dims, ranks);
  const size_t es = f64 ? 8 : 4;
  int64_t off = 0;
  double* pb = c.take<double>(z.Isum);
  double* cb = c.take<double>(z.Isum);
  for (int k = 0; k < N; ++k) {
    d.p[k] = pb ? pb + off : nullptr;
    d.cdf[k] = cb ? cb + off : nullptr;
    off += dims[k];
  }
  d.A = c.take<char>(static_cast<size_t>(J) * z.Lmax * es);
  d.Y = c.take<char>(static_cast<size_t>(J) * z.Imax * es);
  const size_t L2 = static_cast<size_t>(z.Lmax) * z.Lmax;
  d.M = c.take<double>(L2);
  d.BT = c.take<double>(static_cast<size_t>(z.Imax) * z.Lmax);
  d.Lrow = c.take<double>(L2);
  d.Lcol = c.take<double>(L2);
  d.invdiag = c.take<double>(z.Lmax);
  d.keep = c.take<int>(z.Lmax);
  d.info = c.take<int>(1);
  d.limg = c.take<char>(img_bytes(z.Lmax, !f64));
  d.mimg = f64 ? nullptr : reinterpret_cast<float*>(c.take<char>(img_bytes(z.Lmax, true)));
  const size_t n12 = static_cast<size_t>(z.n1) * z.n1;
  d.G1 = c.take<double>(n12);
  d.L1row = c.take<double>(n12);
  d.L1col = c.take<double>(n12);
  d.inv1 = c.take<double>(z.n1);
  d.keep1 = c.take<int>(z.n1);
  d.info1 = c.take<int>(1);
  d.img1 = reinterpret_cast<double*>(c.take<char>(img_bytes(z.n1, false)));
  if (z.n2 > 0) {
    const size_t n22 = static_cast<size_t>(z.n2) * z.n2;
    d.G2 = c.take<double>(n22);
    d.L2row = c.take<double>(n22);
    d.L2col = c.take<double>(n22);
    d.inv2 = c.take<double>(z.n2);
    d.keep2 = c.take<int>(z.n2);
    d.info2 = c.take<int>(1);
    d.img2 = reinterpret_cast<double*>(c.take<char>(img_bytes(z.n2, false)));
  } else {
    d.G2 = d.L2row = d.L2col = d.inv2 = d.img2 = nullptr;
    d.keep2 = d.info2 = nullptr;
  }
  d.ell = c.take<double>(z.Imax);
}

// Streams and events of one batched step's two concurrent branches.
struct StepStreams {
  cudaStream_t main, side;
  cudaEvent_t fork, info, join;
};

// The leverage stages (Gram, Cholesky-QR pass(es), rows with the fused p / CDF step) of
// every instance's current core on one stream; `wait_info` (if set) is waited for before the
// rows, whose CDF step reads the solve's status.
inline cudaError_t issue_leverage(const BLaunch& bl, int step, int init_k, unsigned* err,
                                  cudaStream_t st, cudaEvent_t wait_info) {
  cudaError_t e;
  if ((e = bl_gram(bl, step, init_k, 1, st)) != cudaSuccess) return e;
  if ((e = bl_cholesky(bl, step, init_k, 1, err, st)) != cudaSuccess) return e;
  if (bl.n2max > 0) {
    if ((e = bl_gram(bl, step, init_k, 2, st)) != cudaSuccess) return e;
    if ((e = bl_cholesky(bl, step, init_k, 2, err, st)) != cudaSuccess) return e;
  }
  if (wait_info && (e = cudaStreamWaitEvent(st, wait_info, 0)) != cudaSuccess) return e;
  return bl_leverage_rows(bl, step, init_k, err, st);
}

// One lockstep step of every instance: draws, subchain rows and fibres, normal equations,
// then the LS solve on `main` concurrently with the new distribution (from B^T, which has the
// column space of the new core whenever the normal matrix is nonsingular) on `side`; both
// branches are joined on `main`. A batch that samples uniformly throughout has no
// distribution branch. Under the column-dropping rule the new core's column space is that of
// the kept columns of B^T only, so the distribution is formed from the new core itself,
// after the solve, on `main`.
inline cudaError_t issue_step(const BLaunch& bl, int step, unsigned* err, const StepStreams& s) {
  cudaError_t e;
  if ((e = bl_sample_chain_gather(bl, step, s.main)) != cudaSuccess) return e;
  if ((e = bl_contract(bl, step, s.main)) != cudaSuccess) return e;
  if (!bl.leverage) {   // uniform sampling only: no distribution branch
    if ((e = bl_cholesky(bl, step, 0, 0, err, s.main)) != cudaSuccess) return e;
    return bl_solve(bl, step, s.main);
  }
  if (bl.ls_mode == 1) {
    if ((e = bl_cholesky(bl, step, 0, 0, err, s.main)) != cudaSuccess) return e;
    if ((e = bl_solve(bl, step, s.main)) != cudaSuccess) return e;
    return issue_leverage(bl, step, 0, err, s.main, nullptr);
  }
  if ((e = cudaEventRecord(s.fork, s.main)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s.side, s.fork, 0)) != cudaSuccess) return e;
  if ((e = bl_cholesky(bl, step, 0, 0, err, s.main)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(s.info, s.main)) != cudaSuccess) return e;
  if ((e = bl_solve(bl, step, s.main)) != cudaSuccess) return e;
  if ((e = issue_leverage(bl, step, 0, err, s.side, s.info)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(s.join, s.side)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s.main, s.join, 0);
}

}  // namespace trk
