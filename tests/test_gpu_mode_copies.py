"""The sampled drivers read the fibres of a strided mode from a copy of X with that mode
last (contiguous), made at the start of each call. The copies change only where the bytes
are read from: the drivers' results are bitwise those read from X itself
(TRALS_PERMUTE=0), and both match the oracle as the other parity tests require."""

import pytest
import torch

from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = T.Context(0)
    yield c
    c.close()


def _run(ctx, X, dims, ranks, J, sweeps, prec, init):
    out = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, X, ranks, J, sweeps, 17, prec, out, init_cores=init)
    T.tr_status_sync(ctx)
    return [o.cpu() for o in out]


@pytest.mark.parametrize("dims,ranks,xdt,prec", [
    ((60, 50, 40), (4, 5, 3), torch.float32, T.TR_PREC_MIXED),
    ((60, 50, 40), (4, 5, 3), torch.float64, T.TR_PREC_FP64),
    ((12, 9, 10, 33), (2, 3, 2, 3), torch.float32, T.TR_PREC_MIXED),
    ((37, 41, 29), (3, 3, 3), torch.float32, T.TR_PREC_MIXED),   # odd sizes: ragged tiles
])
def test_copies_give_identical_cores(ctx, monkeypatch, dims, ranks, xdt, prec):
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=3, rel_noise=1e-2, dtype=xdt)
    Xd = X.to(DEV)
    init = [inputs.slice_major(c).to(DEV) for c in inputs.random_cores(dims, ranks, 4)]
    a = _run(ctx, Xd, dims, ranks, 500, 4, prec, init)
    monkeypatch.setenv("TRALS_PERMUTE", "0")
    b = _run(ctx, Xd, dims, ranks, 500, 4, prec, init)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
