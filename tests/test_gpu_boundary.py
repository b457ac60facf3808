"""Error paths of the C ABI on the GPU: an expired bounded device wait (the tensor-core
contraction's pipeline waits, made to expire with a poll limit of 0) returns TR_ERR_TIMEOUT,
leaves the core unchanged and leaves the context usable; a context's own HBM budget is
enforced with TR_ERR_BUDGET before anything is launched."""

import numpy as np
import pytest
import torch

from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _problem(J, L, I, seed):
    g = torch.Generator(device=DEV).manual_seed(seed)
    A = torch.randn((J, L), generator=g, device=DEV)
    Y = A @ torch.randn((L, I), generator=g, device=DEV) + 0.05 * torch.randn(
        (J, I), generator=g, device=DEV)
    return A.contiguous(), Y.contiguous()


def test_expired_wait_reports_timeout_and_keeps_core():
    ctx = T.Context(0)
    try:
        A, Y = _problem(4000, 100, 500, 1)
        ref = torch.empty((500, 10, 10), dtype=torch.float64, device=DEV)
        T.tr_solve(ctx, A, Y, 10, 10, T.TR_PREC_MIXED, ref)
        T.tr_status_sync(ctx)
        assert T.tr_get_wait_limit(ctx) < 0
        T.tr_set_wait_limit(ctx, 0)          # every pipeline wait expires at once
        assert T.tr_get_wait_limit(ctx) == 0
        out = torch.full((500, 10, 10), 2.5, dtype=torch.float64, device=DEV)
        T.tr_solve(ctx, A, Y, 10, 10, T.TR_PREC_MIXED, out)
        with pytest.raises(T.TrError) as e:
            T.tr_status_sync(ctx)
        assert e.value.status == T.TR_ERR_TIMEOUT
        assert torch.all(out == 2.5), "the core was written after an expired wait"
        # the context stays usable: the default limit gives the reference result again
        T.tr_set_wait_limit(ctx, -1)
        T.tr_solve(ctx, A, Y, 10, 10, T.TR_PREC_MIXED, out)
        T.tr_status_sync(ctx)
        assert torch.equal(out, ref)
    finally:
        ctx.close()


def test_expired_wait_in_the_driver():
    dims, ranks = (60, 50, 40), (4, 5, 3)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=3, rel_noise=1e-2, device=DEV)
    init = [inputs.slice_major(c).to(DEV) for c in inputs.random_cores(dims, ranks, 4)]
    ctx = T.Context(0)
    try:
        T.tr_set_wait_limit(ctx, 0)
        out = T.empty_cores(dims, ranks, device=DEV)
        with pytest.raises(T.TrError) as e:
            T.tr_als_sampled(ctx, X, ranks, 600, 2, 5, T.TR_PREC_MIXED, out, init_cores=init)
        assert e.value.status == T.TR_ERR_TIMEOUT
        T.tr_set_wait_limit(ctx, -1)
        T.tr_als_sampled(ctx, X, ranks, 600, 2, 5, T.TR_PREC_MIXED, out, init_cores=init)
    finally:
        ctx.close()
    # the context that met the timeout gives the same cores as a fresh one
    fresh = T.Context(0)
    try:
        ref = T.empty_cores(dims, ranks, device=DEV)
        T.tr_als_sampled(fresh, X, ranks, 600, 2, 5, T.TR_PREC_MIXED, ref, init_cores=init)
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
    finally:
        fresh.close()


def test_context_budget_is_enforced():
    dims, ranks = (200, 200, 200), (10, 10, 10)
    X = torch.zeros(dims, device=DEV)
    ctx = T.Context(0, hbm_budget_bytes=1 << 20)        # 1 MiB: far below the workspace
    try:
        out = T.empty_cores(dims, ranks, device=DEV)
        before = [c.clone() for c in out]
        with pytest.raises(T.TrError) as e:
            T.tr_als_sampled(ctx, X, ranks, 4000, 1, 0, T.TR_PREC_MIXED, out)
        assert e.value.status == T.TR_ERR_BUDGET
        assert "budget" in str(e.value)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(out, before))
        A = torch.zeros((4000, 100), device=DEV)
        Y = torch.zeros((4000, 200), device=DEV)
        core = torch.empty((200, 10, 10), dtype=torch.float64, device=DEV)
        with pytest.raises(T.TrError) as e:
            T.tr_solve(ctx, A, Y, 10, 10, T.TR_PREC_MIXED, core)
        assert e.value.status == T.TR_ERR_BUDGET
    finally:
        ctx.close()
    # the same call fits a context without a cap
    ctx = T.Context(0)
    try:
        A, Y = _problem(400, 16, 30, 9)
        core = torch.empty((30, 4, 4), dtype=torch.float64, device=DEV)
        T.tr_solve(ctx, A, Y, 4, 4, T.TR_PREC_MIXED, core)
        T.tr_status_sync(ctx)
        assert torch.isfinite(core).all()
    finally:
        ctx.close()
