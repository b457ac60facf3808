"""A sample size per sweep (Sec. 4.2; tr_als_sampled_schedule): FP64 sweeps with a growing
schedule match the oracle's, a constant schedule is the scalar call bit for bit, and a bad
entry is refused before any launch."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = T.Context(0)
    yield c
    c.close()


def to_dev_core(core_paper):
    return torch.from_numpy(np.ascontiguousarray(np.transpose(core_paper, (1, 0, 2)))).to(DEV)


def to_paper(core_dev):
    return np.ascontiguousarray(np.transpose(core_dev.cpu().numpy(), (1, 0, 2)))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims,ranks,sched", [((30, 25, 20), (3, 4, 2), [150, 400, 257]),
                                              ((12, 9, 10, 11), (2, 3, 2, 3), [600, 90])])
def test_schedule_matches_oracle_fp64(ctx, dims, ranks, sched):
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=6, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 7)]
    ref = orc.tr_als_sampled(X.numpy(), init, sched, len(sched), 21, solver="normal")
    out = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, X.to(DEV), ranks, sched, len(sched), 21, T.TR_PREC_FP64, out,
                     init_cores=[to_dev_core(c) for c in init])
    for k in range(len(dims)):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8


def test_constant_schedule_is_the_scalar_call(ctx):
    dims, ranks = (40, 30, 20), (4, 4, 4)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=2, rel_noise=1e-2)
    Xd = X.to(DEV)
    init = [inputs.slice_major(c).to(DEV) for c in inputs.random_cores(dims, ranks, 3)]
    a, b = T.empty_cores(dims, ranks), T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, Xd, ranks, 500, 3, 9, T.TR_PREC_MIXED, a, init_cores=init)
    T.tr_als_sampled(ctx, Xd, ranks, [500, 500, 500], 3, 9, T.TR_PREC_MIXED, b, init_cores=init)
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def test_schedule_rejects_a_bad_entry(ctx):
    dims, ranks = (10, 11, 12), (2, 2, 2)
    X = torch.zeros(dims, dtype=torch.float32, device=DEV)
    out = T.empty_cores(dims, ranks)
    with pytest.raises(T.TrError) as e:
        T.tr_als_sampled(ctx, X, ranks, [100, 0], 2, 1, T.TR_PREC_MIXED, out)
    assert e.value.status == T.TR_ERR_INVALID_ARG
