"""Adaptive sample sizes (Sec. 4.2) on the GPU: repeated draws merged into one weighted row
(tr_merge_samples, and the drivers with tr_set_merge_duplicates) and one sample size per core
update (tr_als_sampled_adaptive), against the oracle's merge_duplicates and its per-update
schedule."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_dev_core(c):
    return torch.from_numpy(np.ascontiguousarray(np.transpose(c, (1, 0, 2)))).to(DEV)


def to_paper(c):
    return np.ascontiguousarray(np.transpose(c.cpu().numpy(), (1, 0, 2)))


@pytest.fixture(scope="module")
def ctx():
    c = T.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("dims,J", [((3, 4, 5), 600), ((7, 3, 6, 2), 8192), ((50, 40, 30), 1)])
def test_merge_samples_matches_the_oracle(ctx, dims, J):
    N = len(dims)
    ranks = (2,) * N
    cores = [c.numpy() for c in inputs.random_cores(dims, ranks, 3)]
    ps, cdfs = zip(*[orc.core_distribution(c) for c in cores])
    k = N - 1
    idx_o, w_o = orc.draw_samples(list(ps), list(cdfs), k, J, 9, 4)
    mi, mw, _ = orc.merge_duplicates(idx_o, w_o)
    idx = torch.from_numpy(idx_o.astype(np.int32)).to(DEV)
    w = torch.from_numpy(w_o).to(DEV)
    io = torch.full_like(idx, -1)
    wo = torch.full_like(w, -1.0)
    jo = torch.zeros(1, dtype=torch.int64, device=DEV)
    T.tr_merge_samples(ctx, k, dims, idx, w, io, wo, jo)
    T.tr_status_sync(ctx)
    m = int(jo.item())
    assert m == mi.shape[0]
    np.testing.assert_array_equal(io[:m].cpu().numpy(), mi)
    np.testing.assert_array_equal(wo[:m].cpu().numpy(), mw)
    if m < J:
        assert torch.all(io[m:] == -1) and torch.all(wo[m:] == -1.0)


def test_merge_samples_rejects_oversized_input(ctx):
    J = 8193
    idx = torch.zeros((J, 2), dtype=torch.int32, device=DEV)
    w = torch.ones(J, dtype=torch.float64, device=DEV)
    jo = torch.zeros(1, dtype=torch.int64, device=DEV)
    with pytest.raises(T.TrError) as e:
        T.tr_merge_samples(ctx, 2, (5, 6, 7), idx, w, idx.clone(), w.clone(), jo)
    assert e.value.status == T.TR_ERR_INVALID_ARG


def _case():
    dims, ranks = (6, 7, 8), (2, 3, 2)
    X, true = inputs.tr_plus_noise(dims, ranks, seed=8, rel_noise=1e-2, dtype=torch.float64)
    pert = inputs.random_cores(dims, ranks, 9)
    init = [(t + 0.3 * p).numpy() for t, p in zip(true, pert)]
    return dims, ranks, X, init


def test_merging_driver_matches_the_oracle_fp64(ctx):
    """J = 600 draws over at most 56 cells per update: most draws repeat."""
    dims, ranks, X, init = _case()
    J, sweeps = 600, 3
    ref = orc.tr_als_sampled(X.numpy(), init, J, sweeps, 5, solver="normal", merge=True)
    out = T.empty_cores(dims, ranks)
    T.tr_set_merge_duplicates(ctx, True)
    try:
        T.tr_als_sampled(ctx, X.to(DEV), ranks, J, sweeps, 5, T.TR_PREC_FP64, out,
                         init_cores=[to_dev_core(c) for c in init])
    finally:
        T.tr_set_merge_duplicates(ctx, False)
    for k in range(3):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8


def test_merging_driver_mixed_equals_unmerged(ctx):
    dims, ranks, X, init = _case()
    Xf = X.float().to(DEV)
    a = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, Xf, ranks, 600, 1, 5, T.TR_PREC_MIXED, a,
                     init_cores=[to_dev_core(c) for c in init])
    b = T.empty_cores(dims, ranks)
    T.tr_set_merge_duplicates(ctx, True)
    try:
        T.tr_als_sampled(ctx, Xf, ranks, 600, 1, 5, T.TR_PREC_MIXED, b,
                         init_cores=[to_dev_core(c) for c in init])
    finally:
        T.tr_set_merge_duplicates(ctx, False)
    for x, y in zip(a, b):
        assert rel(y.cpu().numpy(), x.cpu().numpy()) < 1e-4


def test_per_update_sample_sizes_match_the_oracle_fp64(ctx):
    dims, ranks = (20, 18, 16), (3, 4, 2)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=10, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 11)]
    Js = [[300, 420, 250], [380, 260, 510]]
    ref = orc.tr_als_sampled(X.numpy(), init, Js, 2, 12, solver="normal")
    out = T.empty_cores(dims, ranks)
    Xd = X.to(DEV)
    T.tr_als_sampled(ctx, Xd, ranks, Js, 2, 12, T.TR_PREC_FP64, out,
                     init_cores=[to_dev_core(c) for c in init])
    for k in range(3):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8
    # a schedule constant within each sweep is the per-sweep schedule, bit for bit
    a = T.empty_cores(dims, ranks)
    b = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, Xd, ranks, [[300] * 3, [380] * 3], 2, 12, T.TR_PREC_FP64, a,
                     init_cores=[to_dev_core(c) for c in init])
    T.tr_als_sampled(ctx, Xd, ranks, [300, 380], 2, 12, T.TR_PREC_FP64, b,
                     init_cores=[to_dev_core(c) for c in init])
    for x, y in zip(a, b):
        assert torch.equal(x, y)
