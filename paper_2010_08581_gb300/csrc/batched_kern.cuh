// Device helpers shared by the batched stage kernels (batched.cu, batched_chol.cu,
// batched_solve32.cu, batched_solve64.cu, batched_fit.cu): which core each instance
// updates in a step, and the dynamic shared-memory limit of the batched kernels.
#pragma once

#include "batched.cuh"

namespace trk {
namespace {

// The core being updated (or, in an initialisation step, the core whose initial distribution
// is formed) and its sizes. Leverage stages (`lev`) run in both kinds of step; the sampling
// and solve stages only in updates.
struct Cur {
  bool active;
  bool init;
  int n, Rl, Rr, L;
  int64_t I;
  int t;             // update id (step) of an update
};

__device__ __forceinline__ Cur current(const BInst& d, int step, int init_k, bool lev) {
  Cur c{};
  if (lev && d.uniform) return c;   // uniform sampling forms no distributions
  int k = 0, t = step;
  if (d.slot) {
    const SlotState& s = *d.slot;
    if (s.status != kSlotRunning) return c;
    t = s.step;
    if (t < 0) {
      if (!lev) return c;
      k = t + d.N;
    }
  } else if (init_k > 0) {
    if (d.nupd <= 0 || init_k >= d.N) return c;
    k = init_k;
  }
  if (k > 0) {
    c.init = true;
    c.n = k;
  } else {
    if (t >= d.nupd) return c;
    c.n = t % d.N;
    c.t = t;
  }
  c.active = true;
  c.Rl = d.ranks[(c.n - 1 + d.N) % d.N];
  c.Rr = d.ranks[c.n];
  c.L = c.Rl * c.Rr;
  c.I = d.dims[c.n];
  return c;
}

constexpr int kDyn = 200 * 1024;

}  // namespace

// Per-precision halves of bl_solve (batched_solve32.cu / batched_solve64.cu) and the
// attribute set-up of each translation unit.
cudaError_t bl_solve_f32(const BLaunch& b, int step, cudaStream_t st);
cudaError_t bl_solve_f64(const BLaunch& b, int step, cudaStream_t st);
cudaError_t batched_chol_attributes();
cudaError_t batched_solve32_attributes();
cudaError_t batched_solve64_attributes();
cudaError_t batched_fit_attributes();

}  // namespace trk
