"""The LS step's rule for small pivots (tr_set_ls_rank): TR_LS_RANK_DROP gives the oracle's
basic least-squares solution of a rank-deficient design (a repeated and a zero column) in
FP64 and on the mixed path's FP64 branch, batched and single-problem alike; the default
still reports TR_ERR_SINGULAR; unknown rules are refused."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
EPS = 2.220446049250313e-16


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_paper(core_dev):
    return np.ascontiguousarray(np.transpose(core_dev.cpu().numpy(), (1, 0, 2)))


def _deficient(J, Rl, Rr, I, seed):
    rng = np.random.default_rng(seed)
    L = Rl * Rr
    A = rng.standard_normal((J, L))
    A[:, 5] = A[:, 2]
    A[:, L - 1] = 0.0
    Y = A @ rng.standard_normal((L, I)) + 0.05 * rng.standard_normal((J, I))
    return A, Y


@pytest.mark.parametrize("prec", [T.TR_PREC_FP64, T.TR_PREC_MIXED])
def test_drop_gives_the_basic_solution(prec):
    ctx = T.Context(0)
    T.tr_set_ls_rank(ctx, T.TR_LS_RANK_DROP)
    assert T.tr_get_ls_rank(ctx) == T.TR_LS_RANK_DROP
    J, Rl, Rr, I = 600, 4, 4, 37
    A, Y = _deficient(J, Rl, Rr, I, 3)
    dt = torch.float64 if prec == T.TR_PREC_FP64 else torch.float32
    A_in, Y_in = A.astype(np.float32 if dt == torch.float32 else np.float64), \
        Y.astype(np.float32 if dt == torch.float32 else np.float64)
    Z, keep = orc.sampled_ls_normal_drop(A_in.astype(np.float64), Y_in.astype(np.float64),
                                         Rl * Rr * EPS)
    assert list(np.nonzero(~keep)[0]) == [5, Rl * Rr - 1]
    out = torch.empty((I, Rl, Rr), dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, torch.from_numpy(A_in).to(DEV), torch.from_numpy(Y_in).to(DEV), Rl, Rr,
               prec, out)
    T.tr_status_sync(ctx)
    ref = orc.core_from_solution(Z, Rl, Rr)
    assert rel(to_paper(out), ref) < (1e-9 if prec == T.TR_PREC_FP64 else 1e-4)
    ctx.close()


def test_default_still_stops_and_unknown_rules_are_refused():
    ctx = T.Context(0)
    assert T.tr_get_ls_rank(ctx) == T.TR_LS_RANK_STOP
    A, Y = _deficient(300, 4, 4, 9, 4)
    out = torch.full((9, 4, 4), 3.0, dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, torch.from_numpy(A).to(DEV), torch.from_numpy(Y).to(DEV), 4, 4,
               T.TR_PREC_FP64, out)
    with pytest.raises(T.TrError) as e:
        T.tr_status_sync(ctx)
    assert e.value.status == T.TR_ERR_SINGULAR
    assert torch.all(out == 3.0)
    with pytest.raises(T.TrError) as e:
        T.tr_set_ls_rank(ctx, 2)
    assert e.value.status == T.TR_ERR_INVALID_ARG
    ctx.close()


def test_drivers_run_through_rank_deficient_updates():
    """The oscillatory 10-way tensor, whose optimal cores are rank-deficient: with DROP the
    dense and sampled drivers finish without a singular status, and the batched driver gives
    the single driver's cores."""
    ctx = T.Context(0)
    T.tr_set_ls_rank(ctx, T.TR_LS_RANK_DROP)
    dims, ranks = (4,) * 10, (10,) * 10
    X = inputs.oscillatory("linear_growth").to(DEV)
    init = [inputs.slice_major(c).to(DEV) for c in inputs.random_cores(dims, ranks, 77)]
    out = T.empty_cores(dims, ranks)
    T.tr_als(ctx, X, ranks, 8, 0, T.TR_PREC_MIXED, out, init_cores=init)
    e_dense = T.tr_rel_error(ctx, X, ranks, out)
    assert np.isfinite(e_dense)
    T.tr_als_sampled(ctx, X, ranks, 2000, 4, 5, T.TR_PREC_MIXED, out, init_cores=init)
    single = [c.clone() for c in out]
    probs = [dict(X=X, ranks=ranks, J=2000, seed=5, init=True, cores=[c.clone() for c in init])]
    T.tr_als_sampled_batched(ctx, probs, 4, T.TR_PREC_MIXED)
    e_s = T.tr_rel_error(ctx, X, ranks, single)
    e_b = T.tr_rel_error(ctx, X, ranks, probs[0]["cores"])
    assert np.isfinite(e_s) and abs(e_s - e_b) < 0.01 * e_s
    ctx.close()


def _zero_slice_ring(noise=0.0):
    """Noise-free (or noisy) 9 x 8 x 7 ring, ranks 3, whose rank index 2 between cores 0 and
    1 is unused (core 1's first-row slices and core 0's last-column slices are zero), with a
    start near the truth that keeps those slices zero: every update of cores 0 and 1 has a
    design with exactly zero columns."""
    dims, ranks = (9, 8, 7), (3, 3, 3)
    true = [c.numpy() for c in inputs.random_cores(dims, ranks, 21)]
    true[1][2, :, :] = 0.0
    true[0][:, :, 2] = 0.0
    X = np.ascontiguousarray(orc.tr_reconstruct(true))
    if noise:
        rng = np.random.default_rng(23)
        X = np.ascontiguousarray(
            X + noise * np.linalg.norm(X) / np.sqrt(X.size) * rng.standard_normal(X.shape))
    pert = [c.numpy() for c in inputs.random_cores(dims, ranks, 22)]
    init = [t + 0.05 * p for t, p in zip(true, pert)]
    init[1][2, :, :] = 0.0
    init[0][:, :, 2] = 0.0
    return dims, ranks, X, init


def _dev_cores(cores):
    return [torch.from_numpy(np.ascontiguousarray(np.transpose(c, (1, 0, 2)))).to(DEV)
            for c in cores]


def test_drop_driver_matches_the_oracle_fp64():
    """Whole FP64 sweeps under TR_LS_RANK_DROP against the oracle's dropping driver, whose
    next distribution is the leverage of the new core: same draws, cores within 1e-8."""
    dims, ranks, X, init = _zero_slice_ring()
    J, sweeps = 300, 5
    ref = orc.tr_als_sampled(X, init, J, sweeps, 4, solver="normal_drop")
    ctx = T.Context(0)
    try:
        T.tr_set_ls_rank(ctx, T.TR_LS_RANK_DROP)
        out = T.empty_cores(dims, ranks)
        T.tr_als_sampled(ctx, torch.from_numpy(X).to(DEV), ranks, J, sweeps, 4, T.TR_PREC_FP64,
                         out, init_cores=_dev_cores(init))
        for k in range(3):
            assert rel(to_paper(out[k]), ref[k]) < 1e-8, k
    finally:
        ctx.close()


def test_drop_driver_final_error_mixed():
    dims, ranks, X, init = _zero_slice_ring(noise=1e-2)
    J, sweeps = 300, 8
    ref = orc.tr_als_sampled(X, init, J, sweeps, 4, solver="normal_drop")
    e_o = orc.rel_error(ref, X)
    ctx = T.Context(0)
    try:
        T.tr_set_ls_rank(ctx, T.TR_LS_RANK_DROP)
        Xd = torch.from_numpy(X).float().to(DEV)
        out = T.empty_cores(dims, ranks)
        T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, 4, T.TR_PREC_MIXED, out,
                         init_cores=_dev_cores(init))
        e_g = orc.rel_error([to_paper(c) for c in out], X)
        assert abs(e_g - e_o) <= 0.01 * e_o, (e_g, e_o)
        # the batched driver follows the same rule and gives the same cores in FP64
        T.tr_set_ls_rank(ctx, T.TR_LS_RANK_DROP)
        single = T.empty_cores(dims, ranks)
        Xd64 = torch.from_numpy(X).to(DEV)
        T.tr_als_sampled(ctx, Xd64, ranks, J, 3, 4, T.TR_PREC_FP64, single,
                         init_cores=_dev_cores(init))
        probs = [dict(X=Xd64, ranks=ranks, J=J, seed=4, init=True, cores=_dev_cores(init))]
        T.tr_als_sampled_batched(ctx, probs, 3, T.TR_PREC_FP64)
        for a, b in zip(single, probs[0]["cores"]):
            assert rel(b.cpu().numpy(), a.cpu().numpy()) < 1e-10
    finally:
        ctx.close()
