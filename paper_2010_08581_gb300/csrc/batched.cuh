// Batched execution of many independent TR-ALS-Sampled problems (Alg. 2 per instance).
//
// Every stage is one launch for all instances: blockIdx.x selects the instance, blockIdx.y
// a tile of its work, and each CTA reads its instance's sizes and buffers from a
// device-resident table. No CTA ever mixes two instances, so an instance's results do not
// depend on which other instances share the launch.
//
// Instances advance in lockstep "steps": at step t an instance with N modes and
// nupd = sweeps * N updates performs the update of core t % N in sweep t / N with
// update_id t (the same counter the single-problem driver uses), or nothing if t >= nupd.
//
// A served instance (slot != nullptr) keeps its own step counter in device memory instead:
// steps 1-N .. -1 form the initial distributions of cores 1 .. N-1 (Alg. 2 before the first
// sweep), steps t >= 0 are updates as above, and after the last update of each sweep the
// relative fit is evaluated and the stop rule applied on the device. Every launch of a
// serving tick therefore serves slots at different points of their decompositions.
#pragma once

#include "common.cuh"

namespace trk {

constexpr int kMaxServedSweeps = 64;   // sweep cap and fit-history length of a served slot
constexpr int kFitParts = 256;         // partial sums of one fit evaluation (fixed order)

enum SlotStatus : int {
  kSlotIdle = 0,
  kSlotRunning = 1,
  kSlotConverged = 2,   // |fit_s - fit_{s-1}| < tol
  kSlotCapped = 3,      // max_sweeps reached without meeting tol
  kSlotFailed = 4,      // non-finite fit
};

// Device-resident state of one served decomposition.
struct SlotState {
  int step;             // next step (negative: initial distribution of core step + N)
  int status;           // SlotStatus
  int sweeps;           // completed sweeps
  int singular;         // updates whose normal equations were singular (core kept)
  int max_sweeps;
  int pad;
  double tol;           // stop when |fit - fit_prev| < tol (after >= 2 sweeps)
  double fit;           // 1 - ||TR - X||_F / ||X||_F after the last completed sweep
  double fit_prev;
};

struct BInst {
  // problem
  const void* X;                 // row-major data tensor (FP32 or FP64, see xf64)
  int N;
  int xf64;
  int nupd;                      // updates to perform (sweeps * N); 0 = inactive slot
  int draw_init;                 // draw cores 1..N-1 i.i.d. N(0,1) from seed before step 0
  int uniform;                   // uniform sampling (Sec. 5): no distributions, p/cdf unused
  int64_t J;
  uint64_t seed;
  int64_t dims[kMaxModes];
  int64_t stride[kMaxModes];     // row-major element strides of X
  int ranks[kMaxModes];
  double* cores[kMaxModes];      // slice-major [I_k][Rl_k][Rr_k]
  double* p[kMaxModes];
  double* cdf[kMaxModes];
  // per-update scratch
  void* A;                       // J x L_n design rows (FP32 mixed / FP64)
  void* Y;                       // J x I_n fibres
  double* M;                     // L x L normal matrix (FP32-accurate sums in FP64)
  double* BT;                    // I x L right-hand sides (row i = column i of B)
  double* Lrow; double* Lcol; double* invdiag; int* keep; int* info;
  void* limg; float* mimg;       // padded images of the factor and of M for the solves
  // leverage scratch: pass 1 (Gram of the rows' column space), pass 2 (wide modes)
  double* G1; double* L1row; double* L1col; double* inv1; int* keep1; int* info1; double* img1;
  double* G2; double* L2row; double* L2col; double* inv2; int* keep2; int* info2; double* img2;
  double* ell;
  unsigned* counter;
  // serving (nullptr for the batched driver)
  SlotState* slot;
  double* fitp;                  // 2 * kFitParts partial sums of the fit evaluation
  void* fitw;                    // right factors of the fit's mode split (X's precision)
  double* hist;                  // kMaxServedSweeps fits, one per completed sweep
};

// Stage launchers (all instances of `tab[0..count)` in one launch each). `step` is the
// lockstep update counter; for the initial distributions `init_k` > 0 selects core k.
struct BLaunch {
  const BInst* tab;
  int count;
  bool f64;                      // FP64 path (else mixed)
  bool xf64;                     // X is FP64 (else FP32)
  // upper bounds over the instances, for grid sizes
  int64_t Jmax;
  int Lmax;                      // max Rl_k * Rr_k
  int64_t Imax;
  int n1max;                     // max leverage pass-1 Gram size
  int n2max;                     // max leverage pass-2 Gram size (0 if no wide mode)
  // launch shapes (tr_batched_tiles): neither changes any result
  int spw = 4;                   // samples per warp of the sampling kernel, 1..8
  int ctile = 64;                // output tile of the normal-equation contraction, 64 or 32
  bool leverage = true;          // some instance samples by leverage scores (else the
                                 // distribution stages are not launched at all)
  int ls_mode = 0;               // small LS pivots: 0 stop (singular), 1 drop the column
};

cudaError_t bl_init_cores(const BLaunch& b, cudaStream_t st);
cudaError_t bl_sample_chain_gather(const BLaunch& b, int step, cudaStream_t st);
cudaError_t bl_contract(const BLaunch& b, int step, cudaStream_t st);
// which: 0 = normal matrix (solve), 1 = leverage pass 1, 2 = leverage pass 2
cudaError_t bl_cholesky(const BLaunch& b, int step, int init_k, int which, unsigned* err,
                        cudaStream_t st);
cudaError_t bl_solve(const BLaunch& b, int step, cudaStream_t st);
// pass: 1 or 2
cudaError_t bl_gram(const BLaunch& b, int step, int init_k, int pass, cudaStream_t st);
cudaError_t bl_leverage_rows(const BLaunch& b, int step, int init_k, unsigned* err,
                             cudaStream_t st);
// Serving: relative fit of the slots that finished a sweep in this tick, then the stop rule
// and the step counters of all running slots.
cudaError_t bl_fit(const BLaunch& b, unsigned* err, cudaStream_t st);
cudaError_t bl_advance(const BLaunch& b, cudaStream_t st);
cudaError_t batched_attributes();

}  // namespace trk
