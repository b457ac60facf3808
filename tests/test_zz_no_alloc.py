"""tr_solve_noalloc: the least-squares step for callers that cannot allocate device memory
(for example plug-ins inside a host framework that owns all device memory, or serving loops
that must not synchronise the device through cudaMalloc/cudaFree). It runs the same kernels
with the same arguments as tr_solve on a default context, so it must give the same new
core bit for bit, call after call, although every call reuses one fixed scratch array; and
it must not change the device's free memory. This file is collected last so that a failure
here stops a -x run only after all other tests ran."""

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


@pytest.mark.parametrize("prec", [T.TR_PREC_MIXED, T.TR_PREC_FP64])
def test_noalloc_equals_tr_solve_on_consecutive_calls(prec):
    dtype = torch.float32 if prec == T.TR_PREC_MIXED else torch.float64
    ctx = T.Context(0)
    try:
        # consecutive calls with different shapes: a call must not see the previous one's
        # scratch contents
        cases = [(4000, 10, 10, 500, 1), (300, 4, 5, 77, 2), (4000, 10, 10, 500, 3)]
        probs = [_problem(J, Rl, Rr, I, dtype, seed) for (J, Rl, Rr, I, seed) in cases]
        refs, outs, infos = [], [], []
        for (J, Rl, Rr, I, _), (A, Y) in zip(cases, probs):
            ref = torch.empty((I, Rl, Rr), dtype=torch.float64, device=DEV)
            T.tr_solve(ctx, A, Y, Rl, Rr, prec, ref)
            T.tr_status_sync(ctx)
            refs.append(ref)
            outs.append(torch.full((I, Rl, Rr), float("nan"), dtype=torch.float64, device=DEV))
            infos.append(torch.full((1,), -7, dtype=torch.int32, device=DEV))
        torch.cuda.synchronize()
        # first call on this device (address lookup), outside the measured window
        T.tr_solve_noalloc(probs[1][0], probs[1][1], 4, 5, prec, outs[1], infos[1])
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for (J, Rl, Rr, I, _), (A, Y), out, info in zip(cases, probs, outs, infos):
            T.tr_solve_noalloc(A, Y, Rl, Rr, prec, out, info)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        for ref, out, info in zip(refs, outs, infos):
            assert int(info.item()) == 0
            assert torch.equal(out, ref)
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
    # the next call on the same scratch starts from a clean error word
    A2, Y2 = _problem(400, 4, 4, 9, torch.float64, 5)
    out2 = torch.empty((9, 4, 4), dtype=torch.float64, device=DEV)
    T.tr_solve_noalloc(A2, Y2, 4, 4, T.TR_PREC_FP64, out2, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0 and torch.isfinite(out2).all()


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
