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
