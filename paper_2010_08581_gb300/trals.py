"""Thin ctypes binding of ``libtrals.so`` (declared in ``include/trals.h``).

Functions keep the C names and only marshal arguments: torch tensors become device
pointers, per-mode lists become host pointer arrays, and the current torch CUDA stream is
passed as the stream. Every step of the method runs in the library's CUDA kernels; there
is no CPU fallback: loading fails loudly if the library has not been built.
"""

from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtrals.so")

TR_OK, TR_ERR_INVALID_ARG, TR_ERR_OOM, TR_ERR_BUDGET, TR_ERR_SINGULAR, TR_ERR_TIMEOUT, \
    TR_ERR_CUDA, TR_ERR_NOT_CONVERGED = range(8)
TR_F32, TR_F64 = 0, 1
TR_PREC_FP64, TR_PREC_MIXED = 0, 1
TR_SAMPLING_LEVERAGE, TR_SAMPLING_UNIFORM = 0, 1
TR_LS_RANK_STOP, TR_LS_RANK_DROP = 0, 1
TR_FACTOR_DEFAULT, TR_FACTOR_FP64 = 0, 1

_STATUS_NAMES = ["TR_OK", "TR_ERR_INVALID_ARG", "TR_ERR_OOM", "TR_ERR_BUDGET",
                 "TR_ERR_SINGULAR", "TR_ERR_TIMEOUT", "TR_ERR_CUDA", "TR_ERR_NOT_CONVERGED"]

_lib = None

c_int, c_i64, c_u64, c_dbl, c_vp, c_sz = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)
PP = ctypes.POINTER(c_vp)
P64 = ctypes.POINTER(c_i64)
PI = ctypes.POINTER(c_int)

MAX_MODES = 16


class TrInstance(ctypes.Structure):
    """Mirror of ``tr_instance`` in include/trals.h."""
    _fields_ = [("X", c_vp), ("N", c_int), ("dims", c_i64 * MAX_MODES),
                ("ranks", c_int * MAX_MODES), ("J", c_i64), ("seed", c_u64),
                ("cores", c_vp * MAX_MODES), ("init_given", c_int)]


MAX_SERVED_SWEEPS = 64


class TrBatchedTiles(ctypes.Structure):
    """Mirror of ``tr_batched_tiles``."""
    _fields_ = [("samples_per_warp", c_int), ("contract_tile", c_int)]


class TrServerConfig(ctypes.Structure):
    """Mirror of ``tr_server_config``."""
    _fields_ = [("device", c_int), ("hbm_budget_bytes", c_sz), ("arena_bytes", c_sz),
                ("max_slots", c_int), ("max_modes", c_int), ("max_dim", c_i64),
                ("max_rank", c_int), ("max_samples", c_i64), ("max_sweeps", c_int),
                ("fit_tol", c_dbl), ("X_dtype", c_int), ("prec", c_int)]


class TrRequest(ctypes.Structure):
    """Mirror of ``tr_request``."""
    _fields_ = [("X", c_vp), ("N", c_int), ("dims", c_i64 * MAX_MODES),
                ("ranks", c_int * MAX_MODES), ("J", c_i64), ("seed", c_u64),
                ("cores", c_vp * MAX_MODES), ("init_given", c_int), ("max_sweeps", c_int),
                ("fit_tol", c_dbl)]


class TrResult(ctypes.Structure):
    """Mirror of ``tr_result``."""
    _fields_ = [("done", c_int), ("status", c_int), ("sweeps", c_int),
                ("singular_updates", c_int), ("fit", c_dbl), ("fit_change", c_dbl),
                ("t_submit_ns", c_i64), ("t_admit_ns", c_i64), ("t_done_ns", c_i64),
                ("fit_history", c_dbl * MAX_SERVED_SWEEPS)]


class TrServerStats(ctypes.Structure):
    """Mirror of ``tr_server_stats``."""
    _fields_ = [("ticks", c_i64), ("tick_ns", c_i64), ("submitted", c_i64),
                ("completed", c_i64), ("rejected", c_i64), ("updates", c_i64),
                ("active", c_int), ("queued", c_int), ("peak_active", c_int),
                ("charged_bytes", c_sz), ("peak_charged_bytes", c_sz)]


# name -> (restype, argtypes); mirrors include/trals.h
SIGNATURES = {
    "tr_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_sz]),
    "tr_destroy": (None, [c_vp]),
    "tr_last_error": (ctypes.c_char_p, [c_vp]),
    "tr_status_sync": (c_int, [c_vp, c_vp]),
    "tr_leverage": (c_int, [c_vp, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_vp]),
    "tr_leverage_planes": (c_int, [c_vp, c_vp, c_vp, c_i64, c_int, c_vp, c_vp, c_vp, c_vp]),
    "tr_sample": (c_int, [c_vp, c_int, c_int, P64, PP, PP, c_i64, c_u64, c_u64, c_vp, c_vp,
                          c_vp]),
    "tr_sample_uniform": (c_int, [c_vp, c_int, c_int, P64, c_i64, c_u64, c_u64, c_vp, c_vp,
                                  c_vp]),
    "tr_subchain": (c_int, [c_vp, c_int, c_int, P64, PI, PP, c_vp, c_vp, c_i64, c_vp, c_int,
                            c_vp]),
    "tr_gather": (c_int, [c_vp, c_vp, c_int, c_int, P64, c_int, c_vp, c_vp, c_i64, c_vp, c_int,
                          c_vp]),
    "tr_solve": (c_int, [c_vp, c_vp, c_vp, c_int, c_i64, c_int, c_int, c_i64, c_int, c_vp,
                         c_vp]),
    "tr_als_sampled": (c_int, [c_vp, c_vp, c_int, c_int, P64, PI, c_i64, c_int, c_u64, c_int,
                               PP, PP, c_vp]),
    "tr_als": (c_int, [c_vp, c_vp, c_int, c_int, P64, PI, c_int, c_u64, c_int, PP, PP, c_vp]),
    "tr_als_sampled_schedule": (c_int, [c_vp, c_vp, c_int, c_int, P64, PI, P64, c_int, c_u64,
                                        c_int, PP, PP, c_vp]),
    "tr_als_sampled_host": (c_int, [c_vp, c_vp, c_int, c_int, P64, PI, c_i64, c_int, c_u64,
                                    c_int, PP, PP, c_vp]),
    "tr_rel_error": (c_int, [c_vp, c_vp, c_int, c_int, P64, PI, PP, ctypes.POINTER(c_dbl),
                             c_vp]),
    "tr_init_cores": (c_int, [c_vp, c_int, P64, PI, c_u64, c_int, PP, c_vp]),
    "tr_als_sampled_batched": (c_int, [c_vp, ctypes.POINTER(TrInstance), c_int, c_int, c_int,
                                       c_int, c_vp]),
    "tr_solve_noalloc": (c_int, [c_vp, c_vp, c_int, c_i64, c_int, c_int, c_i64, c_int, c_vp,
                                 c_vp, c_vp]),
    "tr_set_ls_rank": (c_int, [c_vp, c_int]),
    "tr_get_ls_rank": (c_int, [c_vp, PI]),
    "tr_set_sampling": (c_int, [c_vp, c_int]),
    "tr_get_sampling": (c_int, [c_vp, PI]),
    "tr_als_sampled_adaptive": (c_int, [c_vp, c_vp, c_int, c_int, P64, PI, P64, c_int, c_u64,
                                        c_int, PP, PP, c_vp]),
    "tr_merge_samples": (c_int, [c_vp, c_int, c_int, P64, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp,
                                 c_vp]),
    "tr_set_merge_duplicates": (c_int, [c_vp, c_int]),
    "tr_get_merge_duplicates": (c_int, [c_vp, PI]),
    "tr_set_factorization": (c_int, [c_vp, c_int]),
    "tr_get_factorization": (c_int, [c_vp, PI]),
    "tr_set_wait_limit": (c_int, [c_vp, c_i64]),
    "tr_get_wait_limit": (c_int, [c_vp, ctypes.POINTER(c_i64)]),
    "tr_set_batched_tiles": (c_int, [c_vp, ctypes.POINTER(TrBatchedTiles)]),
    "tr_get_batched_tiles": (c_int, [c_vp, ctypes.POINTER(TrBatchedTiles)]),
    "tr_server_create": (c_int, [ctypes.POINTER(TrServerConfig), ctypes.POINTER(c_vp)]),
    "tr_server_destroy": (None, [c_vp]),
    "tr_server_last_error": (ctypes.c_char_p, [c_vp]),
    "tr_server_submit": (c_int, [c_vp, ctypes.POINTER(TrRequest), ctypes.POINTER(c_i64)]),
    "tr_server_tick": (c_int, [c_vp, PI]),
    "tr_server_start": (c_int, [c_vp]),
    "tr_server_stop": (c_int, [c_vp]),
    "tr_server_poll": (c_int, [c_vp, c_i64, ctypes.POINTER(TrResult)]),
    "tr_server_wait": (c_int, [c_vp, c_i64, c_i64, ctypes.POINTER(TrResult)]),
    "tr_server_release": (c_int, [c_vp, c_i64]),
    "tr_server_get_stats": (c_int, [c_vp, ctypes.POINTER(TrServerStats)]),
    "tr_profile_begin": (c_int, [c_vp]),
    "tr_profile_end": (c_int, [c_vp, c_vp]),
    "tr_profile_count": (c_int, [c_vp]),
    "tr_profile_entry": (c_int, [c_vp, c_int, ctypes.POINTER(ctypes.c_char_p),
                                 ctypes.POINTER(c_dbl), ctypes.POINTER(c_i64)]),
}


def load():
    """Load libtrals.so (raises if it is missing; nothing falls back to the CPU)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Context:
    """Owns a ``tr_ctx`` (device workspace) on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        lib = load()
        h = c_vp()
        st = lib.tr_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if st != TR_OK:
            raise TrError(st, "tr_create failed: " + (lib.tr_last_error(None) or b"").decode())
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load().tr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int):
        if st != TR_OK:
            raise TrError(st, load().tr_last_error(self.handle).decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_vp(s.cuda_stream)


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return TR_F32
    if t.dtype == torch.float64:
        return TR_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return c_vp(None)
    if t.is_cuda and not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return c_vp(t.data_ptr())


def _ptrs(ts: Sequence[Optional[torch.Tensor]]):
    arr = (c_vp * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr() if t is not None else None
    return ctypes.cast(arr, PP), arr


def _i64s(v):
    arr = (c_i64 * len(v))(*[int(x) for x in v])
    return ctypes.cast(arr, P64), arr


def _ints(v):
    arr = (c_int * len(v))(*[int(x) for x in v])
    return ctypes.cast(arr, PI), arr


def tr_status_sync(ctx: Context, stream=None):
    ctx.check(load().tr_status_sync(ctx.handle, _stream(stream)))


def tr_leverage(ctx: Context, core: torch.Tensor, p: torch.Tensor, cdf: torch.Tensor, stream=None):
    """core: float64 (I, Rl, Rr) slice-major on the device; p, cdf: float64 (I,)."""
    I, Rl, Rr = core.shape
    ctx.check(load().tr_leverage(ctx.handle, _ptr(core), I, Rl, Rr, _ptr(p), _ptr(cdf),
                                 _stream(stream)))


def tr_leverage_planes(ctx: Context, A_hi: torch.Tensor, A_lo: torch.Tensor, p: torch.Tensor,
                       cdf: torch.Tensor, branch: Optional[torch.Tensor] = None, stream=None):
    """A_hi, A_lo: float32 (I, L) row-major on the device (A = A_hi + A_lo); p, cdf: float64
    (I,); branch (optional): int32 (1,) receiving 0 (preconditioned form) or 1 (fallback)."""
    I, L = A_hi.shape
    ctx.check(load().tr_leverage_planes(ctx.handle, _ptr(A_hi), _ptr(A_lo), I, L, _ptr(p),
                                        _ptr(cdf), _ptr(branch) if branch is not None else None,
                                        _stream(stream)))


def tr_sample(ctx: Context, k: int, dims, ps: List[torch.Tensor], cdfs: List[torch.Tensor],
              J: int, seed: int, update_id: int, idx: torch.Tensor, w: torch.Tensor, stream=None):
    N = len(dims)
    d, _d = _i64s(dims)
    pp, _p = _ptrs(ps)
    cp, _c = _ptrs(cdfs)
    ctx.check(load().tr_sample(ctx.handle, N, k, d, pp, cp, J, seed, update_id, _ptr(idx),
                               _ptr(w), _stream(stream)))


def tr_sample_uniform(ctx: Context, k: int, dims, J: int, seed: int, update_id: int,
                      idx: torch.Tensor, w: torch.Tensor, stream=None):
    """Uniform draws (Sec. 5 variant): idx int32 (J, N-1) ring order, w float64 (J,)."""
    N = len(dims)
    d, _d = _i64s(dims)
    ctx.check(load().tr_sample_uniform(ctx.handle, N, k, d, J, seed, update_id, _ptr(idx),
                                       _ptr(w), _stream(stream)))


def tr_set_sampling(ctx: Context, sampling: int):
    """TR_SAMPLING_LEVERAGE or TR_SAMPLING_UNIFORM for the context's driver calls."""
    ctx.check(load().tr_set_sampling(ctx.handle, int(sampling)))


def tr_set_ls_rank(ctx: Context, rule: int):
    """TR_LS_RANK_STOP (default) or TR_LS_RANK_DROP for the context's LS steps."""
    ctx.check(load().tr_set_ls_rank(ctx.handle, int(rule)))


def tr_get_ls_rank(ctx: Context) -> int:
    v = c_int()
    ctx.check(load().tr_get_ls_rank(ctx.handle, ctypes.byref(v)))
    return int(v.value)


def tr_get_sampling(ctx: Context) -> int:
    v = c_int()
    ctx.check(load().tr_get_sampling(ctx.handle, ctypes.byref(v)))
    return int(v.value)


def tr_merge_samples(ctx: Context, k: int, dims, idx: torch.Tensor, w: torch.Tensor,
                     idx_out: torch.Tensor, w_out: torch.Tensor, J_out: torch.Tensor,
                     stream=None):
    """Merge repeated draws (Sec. 4.2): J_out is a device int64 tensor of one element."""
    d, _d = _i64s(list(dims))
    ctx.check(load().tr_merge_samples(ctx.handle, len(dims), k, d, _ptr(idx), _ptr(w),
                                      idx.shape[0], _ptr(idx_out), _ptr(w_out), _ptr(J_out),
                                      _stream(stream)))


def tr_set_merge_duplicates(ctx: Context, on: bool):
    ctx.check(load().tr_set_merge_duplicates(ctx.handle, 1 if on else 0))


def tr_get_merge_duplicates(ctx: Context) -> bool:
    v = c_int()
    ctx.check(load().tr_get_merge_duplicates(ctx.handle, ctypes.byref(v)))
    return bool(v.value)


def tr_set_factorization(ctx: Context, f: int):
    """TR_FACTOR_DEFAULT or TR_FACTOR_FP64 for the mixed path's factorisations."""
    ctx.check(load().tr_set_factorization(ctx.handle, int(f)))


def tr_get_factorization(ctx: Context) -> int:
    v = c_int()
    ctx.check(load().tr_get_factorization(ctx.handle, ctypes.byref(v)))
    return int(v.value)


def tr_set_wait_limit(ctx: Context, polls: int):
    """Polls per bounded wait of the tensor-core contraction (< 0: the default; 0: every
    wait expires at once)."""
    ctx.check(load().tr_set_wait_limit(ctx.handle, int(polls)))


def tr_get_wait_limit(ctx: Context) -> int:
    v = c_i64()
    ctx.check(load().tr_get_wait_limit(ctx.handle, ctypes.byref(v)))
    return int(v.value)


def tr_subchain(ctx: Context, k: int, dims, ranks, cores: List[torch.Tensor], idx: torch.Tensor,
                w: Optional[torch.Tensor], A: torch.Tensor, stream=None):
    N = len(dims)
    d, _d = _i64s(dims)
    r, _r = _ints(ranks)
    cp, _c = _ptrs(cores)
    ctx.check(load().tr_subchain(ctx.handle, N, k, d, r, cp, _ptr(idx), _ptr(w), idx.shape[0],
                                 _ptr(A), _dt(A), _stream(stream)))


def tr_gather(ctx: Context, X: torch.Tensor, k: int, idx: torch.Tensor, w: Optional[torch.Tensor],
              Y: torch.Tensor, stream=None):
    dims = list(X.shape)
    d, _d = _i64s(dims)
    ctx.check(load().tr_gather(ctx.handle, _ptr(X), _dt(X), len(dims), d, k, _ptr(idx), _ptr(w),
                               idx.shape[0], _ptr(Y), _dt(Y), _stream(stream)))


def tr_solve(ctx: Context, A: torch.Tensor, Y: torch.Tensor, Rl: int, Rr: int, prec: int,
             core_out: torch.Tensor, stream=None):
    J, L = A.shape
    I = Y.shape[1]
    ctx.check(load().tr_solve(ctx.handle, _ptr(A), _ptr(Y), _dt(A), J, Rl, Rr, I, prec,
                              _ptr(core_out), _stream(stream)))


def tr_solve_noalloc(A: torch.Tensor, Y: torch.Tensor, Rl: int, Rr: int, prec: int,
                     core_out: torch.Tensor, info: Optional[torch.Tensor] = None, stream=None):
    """tr_solve without any device allocation (fixed 16 MiB library scratch; no context)."""
    lib = load()
    J, L = A.shape
    I = Y.shape[1]
    st = lib.tr_solve_noalloc(_ptr(A), _ptr(Y), _dt(A), J, Rl, Rr, I, prec, _ptr(core_out),
                              _ptr(info), _stream(stream))
    if st != TR_OK:
        raise TrError(st, (lib.tr_last_error(None) or b"").decode())


def tr_init_cores(ctx: Context, dims, ranks, seed: int, k_begin: int, cores, stream=None):
    d, _d = _i64s(dims)
    r, _r = _ints(ranks)
    cp, _c = _ptrs(cores)
    ctx.check(load().tr_init_cores(ctx.handle, len(dims), d, r, seed, k_begin, cp,
                                   _stream(stream)))


def tr_als_sampled(ctx: Context, X: torch.Tensor, ranks, J, sweeps: int, seed: int,
                   prec: int, cores: List[torch.Tensor],
                   init_cores: Optional[List[Optional[torch.Tensor]]] = None, stream=None):
    """J: one sample size, a list with one per sweep (tr_als_sampled_schedule), or a list of
    per-sweep lists with one per core update (tr_als_sampled_adaptive)."""
    dims = list(X.shape)
    d, _d = _i64s(dims)
    r, _r = _ints(ranks)
    cp, _c = _ptrs(cores)
    if init_cores is not None:
        ip, _i = _ptrs(init_cores)
    else:
        ip = ctypes.cast(c_vp(None), PP)
    if isinstance(J, (list, tuple)) and J and isinstance(J[0], (list, tuple)):
        flat = [int(v) for row in J for v in row]
        js, _j = _i64s(flat)
        ctx.check(load().tr_als_sampled_adaptive(ctx.handle, _ptr(X), _dt(X), len(dims), d, r,
                                                 js, sweeps, seed, prec, ip, cp,
                                                 _stream(stream)))
        return
    if isinstance(J, (list, tuple)):
        js, _j = _i64s(J)
        ctx.check(load().tr_als_sampled_schedule(ctx.handle, _ptr(X), _dt(X), len(dims), d, r,
                                                 js, sweeps, seed, prec, ip, cp,
                                                 _stream(stream)))
        return
    ctx.check(load().tr_als_sampled(ctx.handle, _ptr(X), _dt(X), len(dims), d, r, J, sweeps,
                                    seed, prec, ip, cp, _stream(stream)))


def tr_als(ctx: Context, X: torch.Tensor, ranks, sweeps: int, seed: int, prec: int,
           cores: List[torch.Tensor], init_cores: Optional[List[Optional[torch.Tensor]]] = None,
           stream=None):
    """Dense TR-ALS (Alg. 1): every row of each least-squares problem, weight 1."""
    dims = list(X.shape)
    d, _d = _i64s(dims)
    r, _r = _ints(ranks)
    cp, _c = _ptrs(cores)
    if init_cores is not None:
        ip, _i = _ptrs(init_cores)
    else:
        ip = ctypes.cast(c_vp(None), PP)
    ctx.check(load().tr_als(ctx.handle, _ptr(X), _dt(X), len(dims), d, r, sweeps, seed, prec,
                            ip, cp, _stream(stream)))


def tr_als_sampled_host(ctx: Context, X_host: torch.Tensor, ranks, J: int, sweeps: int,
                        seed: int, prec: int, cores_host: List[torch.Tensor],
                        init_cores_host: Optional[List[Optional[torch.Tensor]]] = None,
                        stream=None):
    """X_host and cores_host are CPU tensors (pinned for speed)."""
    dims = list(X_host.shape)
    d, _d = _i64s(dims)
    r, _r = _ints(ranks)
    cp, _c = _ptrs(cores_host)
    if init_cores_host is not None:
        ip, _i = _ptrs(init_cores_host)
    else:
        ip = ctypes.cast(c_vp(None), PP)
    ctx.check(load().tr_als_sampled_host(ctx.handle, c_vp(X_host.data_ptr()), _dt(X_host),
                                         len(dims), d, r, J, sweeps, seed, prec, ip, cp,
                                         _stream(stream)))


def tr_als_sampled_batched(ctx: Context, problems, sweeps: int, prec: int, stream=None):
    """problems: list of dicts with keys X (device tensor), ranks, J, seed, cores (list of
    device FP64 (I, Rl, Rr) tensors receiving the result) and optional init (bool: the
    cores already hold the initial cores). All X share one dtype."""
    arr = (TrInstance * len(problems))()
    dt = None
    for i, pr in enumerate(problems):
        X = pr["X"]
        dt = _dt(X) if dt is None else dt
        if _dt(X) != dt:
            raise TypeError("all X of a batch must share one dtype")
        inst = arr[i]
        inst.X = X.data_ptr()
        inst.N = X.ndim
        for k, d in enumerate(X.shape):
            inst.dims[k] = int(d)
            inst.ranks[k] = int(pr["ranks"][k])
            inst.cores[k] = pr["cores"][k].data_ptr()
        inst.J = int(pr["J"])
        inst.seed = int(pr["seed"])
        inst.init_given = 1 if pr.get("init", False) else 0
    ctx.check(load().tr_als_sampled_batched(ctx.handle, arr, len(problems), dt, sweeps, prec,
                                            _stream(stream)))


def tr_set_batched_tiles(ctx: Context, samples_per_warp: int, contract_tile: int):
    t = TrBatchedTiles(int(samples_per_warp), int(contract_tile))
    ctx.check(load().tr_set_batched_tiles(ctx.handle, ctypes.byref(t)))


def tr_get_batched_tiles(ctx: Context):
    t = TrBatchedTiles()
    ctx.check(load().tr_get_batched_tiles(ctx.handle, ctypes.byref(t)))
    return int(t.samples_per_warp), int(t.contract_tile)


def tr_rel_error(ctx: Context, X: torch.Tensor, ranks, cores: List[torch.Tensor], stream=None):
    dims = list(X.shape)
    d, _d = _i64s(dims)
    r, _r = _ints(ranks)
    cp, _c = _ptrs(cores)
    out = c_dbl(0.0)
    ctx.check(load().tr_rel_error(ctx.handle, _ptr(X), _dt(X), len(dims), d, r, cp,
                                  ctypes.byref(out), _stream(stream)))
    return out.value


def tr_profile_begin(ctx: Context):
    ctx.check(load().tr_profile_begin(ctx.handle))


def tr_profile_end(ctx: Context, stream=None):
    """Stop recording; returns {kernel: (total_ms, launches)}."""
    lib = load()
    ctx.check(lib.tr_profile_end(ctx.handle, _stream(stream)))
    out = {}
    for i in range(lib.tr_profile_count(ctx.handle)):
        name, ms, n = ctypes.c_char_p(), c_dbl(), c_i64()
        ctx.check(lib.tr_profile_entry(ctx.handle, i, ctypes.byref(name), ctypes.byref(ms),
                                       ctypes.byref(n)))
        out[name.value.decode()] = (ms.value, n.value)
    return out


def empty_cores(dims, ranks, device="cuda"):
    """Device buffers for the cores, FP64 slice-major (I_k, Rl_k, Rr_k)."""
    N = len(dims)
    return [torch.empty((dims[k], ranks[(k - 1) % N], ranks[k]), dtype=torch.float64,
                        device=device) for k in range(N)]


def _result_dict(r: TrResult):
    n = min(int(r.sweeps), MAX_SERVED_SWEEPS)
    return dict(done=bool(r.done), status=int(r.status), sweeps=int(r.sweeps),
                singular_updates=int(r.singular_updates), fit=float(r.fit),
                fit_change=float(r.fit_change), t_submit_ns=int(r.t_submit_ns),
                t_admit_ns=int(r.t_admit_ns), t_done_ns=int(r.t_done_ns),
                fit_history=[float(r.fit_history[i]) for i in range(n)])


class Server:
    """Owns a ``tr_server``: continuous batching of decomposition requests on one device.

    ``submit`` keeps references to the request's X and core tensors until ``release``."""

    def __init__(self, *, device: int = 0, hbm_budget_bytes: int = 150 << 30,
                 arena_bytes: Optional[int] = None, max_slots: int = 64, max_modes: int = 5,
                 max_dim: int = 1024, max_rank: int = 16, max_samples: int = 2560,
                 max_sweeps: int = 30, fit_tol: float = 1e-4, X_dtype: int = TR_F32,
                 prec: int = TR_PREC_MIXED):
        lib = load()
        cfg = TrServerConfig()
        cfg.device = int(device)
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.arena_bytes = int(arena_bytes if arena_bytes is not None
                              else min(hbm_budget_bytes, 8 << 30))
        cfg.max_slots = int(max_slots)
        cfg.max_modes = int(max_modes)
        cfg.max_dim = int(max_dim)
        cfg.max_rank = int(max_rank)
        cfg.max_samples = int(max_samples)
        cfg.max_sweeps = int(max_sweeps)
        cfg.fit_tol = float(fit_tol)
        cfg.X_dtype = int(X_dtype)
        cfg.prec = int(prec)
        h = c_vp()
        st = lib.tr_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != TR_OK:
            raise TrError(st, "tr_server_create failed: "
                          + (lib.tr_server_last_error(None) or b"").decode())
        self.handle = h
        self.config = cfg
        self._refs = {}

    def _check(self, st: int):
        if st != TR_OK:
            raise TrError(st, (load().tr_server_last_error(self.handle) or b"").decode())

    def submit(self, X: torch.Tensor, ranks, J: int, seed: int, cores: List[torch.Tensor],
               init_given: bool = False, max_sweeps: int = 0, fit_tol: float = -1.0) -> int:
        req = TrRequest()
        req.X = X.data_ptr()
        req.N = X.ndim
        for k, d in enumerate(X.shape):
            req.dims[k] = int(d)
            req.ranks[k] = int(ranks[k])
            req.cores[k] = cores[k].data_ptr()
        req.J = int(J)
        req.seed = int(seed)
        req.init_given = 1 if init_given else 0
        req.max_sweeps = int(max_sweeps)
        req.fit_tol = float(fit_tol)
        t = c_i64()
        self._check(load().tr_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._refs[t.value] = (X, list(cores))
        return t.value

    def tick(self) -> int:
        a = c_int()
        self._check(load().tr_server_tick(self.handle, ctypes.byref(a)))
        return a.value

    def start(self):
        self._check(load().tr_server_start(self.handle))

    def stop(self):
        self._check(load().tr_server_stop(self.handle))

    def poll(self, ticket: int):
        r = TrResult()
        self._check(load().tr_server_poll(self.handle, int(ticket), ctypes.byref(r)))
        return _result_dict(r)

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        r = TrResult()
        self._check(load().tr_server_wait(self.handle, int(ticket), int(timeout_ms),
                                          ctypes.byref(r)))
        return _result_dict(r)

    def release(self, ticket: int):
        self._check(load().tr_server_release(self.handle, int(ticket)))
        self._refs.pop(int(ticket), None)

    def stats(self):
        s = TrServerStats()
        self._check(load().tr_server_get_stats(self.handle, ctypes.byref(s)))
        return {name: int(getattr(s, name)) for name, _ in TrServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().tr_server_destroy(self.handle)
            self.handle = None
            self._refs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
