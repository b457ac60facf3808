// tr_solve_noalloc: the least-squares step of tr_solve (Alg. 2) for callers that cannot
// allocate device memory. Its scratch space is one file-scope device array of fixed size;
// the function never calls cudaMalloc, cudaFree or any allocating library routine.
#include <mutex>
#include <string>

#include "common.cuh"

namespace trk {
// Declared in api.cu: the message returned by tr_last_error(NULL).
void set_global_error(const std::string& msg);
}  // namespace trk

namespace {

using namespace trk;

// 16 MiB of scratch. Every GPU on which the library is loaded holds this array until the
// process exits. All calls share it and it keeps the previous call's contents.
constexpr size_t kScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_solve_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
char* g_scratch_dev[kMaxDevices] = {};

struct Bump {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct Layout {
  void* partial; double* M; double* BT; double* Lrow; double* Lcol; double* invdiag;
  int* keep; int* info; void* limg; float* mimg; float* wimg; unsigned* err; int* fast;
  int splits;
};

// The scratch of one call, carved as tr_solve carves its workspace: the contraction's split
// partials, M, B^T, the factor (row- and column-major), its inverse diagonal and pivot flags,
// the factor's padded image in the solve's arithmetic type, M's FP32 image and the factor's
// FP32 inverse (mixed path), the error word and the flag of the one-CTA factor-and-inverse.
size_t layout(char* base, int64_t J, int L, int64_t I, bool f64, Layout* s) {
  Bump b{base};
  const size_t pbytes = f64 ? normal_eq_workspace(J, L, I, true, &s->splits)
                            : normal_eq_tc_workspace(J, L, I, &s->splits);
  s->partial = b.take<char>(pbytes);
  s->M = b.take<double>(static_cast<size_t>(L) * L);
  s->BT = b.take<double>(static_cast<size_t>(I) * L);
  s->Lrow = b.take<double>(static_cast<size_t>(L) * L);
  s->Lcol = b.take<double>(static_cast<size_t>(L) * L);
  s->invdiag = b.take<double>(L);
  s->keep = b.take<int>(L);
  s->info = b.take<int>(1);
  s->limg = b.take<char>(trsm_image_bytes(L, !f64));
  s->mimg = f64 ? nullptr : reinterpret_cast<float*>(b.take<char>(trsm_image_bytes(L, true)));
  s->wimg = f64 ? nullptr : reinterpret_cast<float*>(b.take<char>(trsm_image_bytes(L, true)));
  s->err = b.take<unsigned>(1);
  s->fast = f64 ? nullptr : b.take<int>(1);
  return b.off;
}

tr_status fail(tr_status st, const std::string& msg) {
  set_global_error("tr_solve_noalloc: " + msg);
  return st;
}

// Once per device, with that device current: resolve the device address of the scratch
// array (host code may not use the symbol itself) and set the kernels' shared-memory
// limits. The address is cached per device ordinal for the life of the process; a device
// reset (cudaDeviceReset) reloads the module and invalidates it (see trals.h).
tr_status setup(int dev, char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_dev[dev]) {
    *out = g_scratch_dev[dev];
    return TR_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
  if (e != cudaSuccess || !p)
    return fail(TR_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
  const char* which = "";
  e = init_kernel_attributes(&which);
  if (e != cudaSuccess)
    return fail(TR_ERR_CUDA, std::string("cudaFuncSetAttribute(") + which + ") failed: " +
                                 cudaGetErrorString(e));
  g_scratch_dev[dev] = static_cast<char*>(p);
  *out = g_scratch_dev[dev];
  return TR_OK;
}

}  // namespace

extern "C" tr_status tr_solve_noalloc(const void* A, const void* Y, tr_dtype dtype, int64_t J,
                                      int Rl, int Rr, int64_t I, tr_precision prec,
                                      double* core_out, int32_t* info, tr_stream stream) {
  if (!A || !Y || !core_out) return fail(TR_ERR_INVALID_ARG, "null pointer");
  if (J < 1 || I < 1 || Rl < 1 || Rr < 1 || Rl * Rr > kMaxL)
    return fail(TR_ERR_INVALID_ARG, "bad sizes");
  if (prec == TR_PREC_FP64 ? dtype != TR_F64 : (prec != TR_PREC_MIXED || dtype != TR_F32))
    return fail(TR_ERR_INVALID_ARG, "TR_PREC_FP64 needs FP64 A/Y, TR_PREC_MIXED FP32 A/Y");
  const bool f64 = prec == TR_PREC_FP64;
  const int L = Rl * Rr;
  Layout s{};
  const size_t need = layout(nullptr, J, L, I, f64, &s);
  if (need > kScratchBytes)
    return fail(TR_ERR_INVALID_ARG,
                "problem needs " + std::to_string(need) + " scratch bytes, more than the fixed " +
                    std::to_string(kScratchBytes));
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(TR_ERR_CUDA, "no current CUDA device");
  }
  char* base = nullptr;
  tr_status st0 = setup(dev, &base);
  if (st0 != TR_OK) return st0;
  layout(base, J, L, I, f64, &s);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t ld = L + I;
  const double eps = 2.220446049250313e-16, eps32 = 1.1920928955078125e-07;
  // The array keeps the previous call's contents: clear the error word first.
  cudaError_t e = cudaMemsetAsync(s.err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    if (f64)
      e = launch_normal_eq(A, Y, true, J, L, I, s.partial, s.splits, st);
    else
      e = launch_normal_eq_tc(static_cast<const float*>(A), static_cast<const float*>(Y), J, L,
                              I, static_cast<float*>(s.partial), s.splits, s.err, st);
  }
  // The same reduction, factorisation and solves as tr_solve (stop-on-singular rule): on the
  // mixed path the reduction also writes M's FP32 work array and image for the FP32 factor.
  ReduceSplit sp;
  const bool pre = !f64 && L >= 4 && L <= 160;
  const bool tiles = !f64 && L >= 4 && L <= 128;   // as tr_solve's default factorisation
  if (pre) {
    sp.hi = reinterpret_cast<float*>(s.Lrow);
    sp.lda = (L + 3) & ~3;
    sp.img = s.mimg;
    sp.np = L + 1;
  }
  if (e == cudaSuccess)
    e = launch_reduce(s.partial, !f64, s.splits, L * ld, ld, L, ld, L, s.M, L, s.BT, L, st, sp);
  if (e == cudaSuccess) {
    if (f64)
      e = launch_cholesky(s.M, L, 0, static_cast<double>(L) * eps, s.Lrow, s.Lcol, s.invdiag,
                          s.keep, s.info, s.err, st, static_cast<double*>(s.limg));
    else
      e = launch_cholesky_mixed(s.M, L, 0, static_cast<double>(L) * eps,
                                static_cast<double>(L) * eps32, s.Lrow, s.Lcol, s.invdiag,
                                s.keep, s.info, s.err, st, static_cast<float*>(s.limg), s.mimg,
                                pre ? reinterpret_cast<float*>(s.Lrow) : nullptr, s.wimg,
                                tiles ? s.fast : nullptr);
  }
  if (e == cudaSuccess) {
    if (!f64 && solve_inv_fits(L))
      e = launch_solve_inv(L, static_cast<const float*>(s.limg), s.mimg, s.invdiag, s.info, I,
                           s.BT, L, Rl, Rr, core_out, s.wimg, st, tiles ? s.fast : nullptr);
    else
      e = launch_trsm(f64 ? 1 : 2, !f64, L, s.Lrow, s.Lcol, s.invdiag, s.info, I, s.BT, L, s.M,
                      Rl, Rr, core_out, nullptr, st, s.limg, s.mimg);
  }
  if (e == cudaSuccess && info)
    e = cudaMemcpyAsync(info, s.info, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fail(TR_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  return TR_OK;
}
