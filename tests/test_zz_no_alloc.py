"""tr_solve_noalloc: the least-squares step for callers that cannot allocate device memory
(for example code running while a CUDA graph is captured in global mode, or serving loops
that must not synchronise the device through cudaMalloc/cudaFree). It must give the same
new core as tr_solve, call after call, although every call reuses one fixed scratch
array. This file is collected last so that a failure here stops a -x run only after all
other tests ran."""

import numpy as np
import pytest
import torch

from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _problem(J, Rl, Rr, I, dtype, seed):
    g = torch.Generator(device=DEV).manual_seed(seed)
    L = Rl * Rr
    A = torch.randn((J, L), generator=g, device=DEV, dtype=torch.float64)
    Y = A @ torch.randn((L, I), generator=g, device=DEV, dtype=torch.float64)
    Y += 0.05 * torch.randn((J, I), generator=g, device=DEV, dtype=torch.float64)
    return A.to(dtype).contiguous(), Y.to(dtype).contiguous()


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("prec", [T.TR_PREC_MIXED, T.TR_PREC_FP64])
def test_noalloc_matches_tr_solve_on_consecutive_calls(prec):
    dtype = torch.float32 if prec == T.TR_PREC_MIXED else torch.float64
    tol = 1e-4 if prec == T.TR_PREC_MIXED else 1e-10
    ctx = T.Context(0)
    try:
        # two calls in a row with different shapes: the second must not see the first's
        # scratch contents
        for (J, Rl, Rr, I, seed) in [(4000, 10, 10, 500, 1), (300, 4, 5, 77, 2),
                                     (4000, 10, 10, 500, 3)]:
            A, Y = _problem(J, Rl, Rr, I, dtype, seed)
            ref = torch.empty((I, Rl, Rr), dtype=torch.float64, device=DEV)
            T.tr_solve(ctx, A, Y, Rl, Rr, prec, ref)
            T.tr_status_sync(ctx)
            out = torch.full((I, Rl, Rr), float("nan"), dtype=torch.float64, device=DEV)
            info = torch.full((1,), -1, dtype=torch.int32, device=DEV)
            T.tr_solve_noalloc(A, Y, Rl, Rr, prec, out, info)
            torch.cuda.synchronize()
            assert int(info.item()) == 0
            assert torch.isfinite(out).all()
            assert _rel(out, ref) <= tol
    finally:
        ctx.close()


def test_noalloc_singular_system_leaves_core_unchanged():
    A, Y = _problem(5, 4, 4, 9, torch.float64, 4)        # J < L: singular normal matrix
    out = torch.full((9, 4, 4), 3.0, dtype=torch.float64, device=DEV)
    info = torch.zeros((1,), dtype=torch.int32, device=DEV)
    T.tr_solve_noalloc(A, Y, 4, 4, T.TR_PREC_FP64, out, info)
    torch.cuda.synchronize()
    assert int(info.item()) > 0
    assert torch.all(out == 3.0)


def test_noalloc_rejects_problems_larger_than_its_scratch():
    J, Rl, Rr, I = 40000, 16, 16, 2000                  # needs far more than 16 MiB
    A = torch.zeros((J, Rl * Rr), dtype=torch.float32, device=DEV)
    Y = torch.zeros((J, I), dtype=torch.float32, device=DEV)
    out = torch.full((I, Rl, Rr), 5.0, dtype=torch.float64, device=DEV)
    with pytest.raises(T.TrError) as e:
        T.tr_solve_noalloc(A, Y, Rl, Rr, T.TR_PREC_MIXED, out)
    assert e.value.status == T.TR_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
    torch.cuda.synchronize()
    assert torch.all(out == 5.0)
