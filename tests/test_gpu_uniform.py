"""Uniform sampling, the Sec. 5 alternative to leverage scores, through the C ABI: draws
bit-exact against the oracle, FP64 sweeps of the single-problem and batched drivers within
1e-8 of the oracle per core, the mixed path within 1 % of the oracle's final error, and the
context's sampling switch (refuses unknown values, and switching back restores the
leverage-score result bit for bit)."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture
def ctx():
    c = T.Context(0)
    T.tr_set_sampling(c, T.TR_SAMPLING_UNIFORM)
    yield c
    c.close()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev_core(core_paper):
    return torch.from_numpy(np.ascontiguousarray(np.transpose(core_paper, (1, 0, 2)))).to(DEV)


def to_paper(core_dev):
    return np.ascontiguousarray(np.transpose(core_dev.cpu().numpy(), (1, 0, 2)))


def np_cores(dims, ranks, seed):
    return [c.numpy() for c in inputs.random_cores(dims, ranks, seed)]


@pytest.mark.parametrize("dims,n,J", [((7, 300, 5), 0, 1), ((50, 40, 30), 1, 4001),
                                      ((3, 4, 5, 6, 7), 2, 1000), ((200, 2), 0, 777),
                                      ((1, 2 ** 31 - 1, 3), 0, 333),
                                      ((500, 500, 500), 2, 4000)])
def test_uniform_draws_bit_exact(ctx, dims, n, J):
    seed, uid = 12345678901, 2 ** 33 + 5
    idx_o, w_o = orc.draw_samples_uniform(dims, n, J, seed, uid)
    idx = torch.empty((J, len(dims) - 1), dtype=torch.int32, device=DEV)
    w = torch.empty(J, dtype=torch.float64, device=DEV)
    T.tr_sample_uniform(ctx, n, dims, J, seed, uid, idx, w)
    T.tr_status_sync(ctx)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    np.testing.assert_array_equal(w.cpu().numpy(), w_o)


@pytest.mark.parametrize("dims,ranks", [((30, 25, 20), (3, 4, 2)), ((12, 9, 10, 11), (2, 3, 2, 3)),
                                        ((40, 6, 33), (4, 3, 5))])
def test_uniform_sweeps_match_oracle_fp64(ctx, dims, ranks):
    """Two FP64 sweeps of the driver with uniform draws against the oracle's Alg. 2 with the
    Sec. 5 uniform sampler and the normal-equation solve."""
    J, sweeps, seed = 300, 2, 21
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=6, rel_noise=1e-2, dtype=torch.float64)
    init = np_cores(dims, ranks, 7)
    ref = orc.tr_als_sampled(X.numpy(), init, J, sweeps, seed, solver="normal",
                             sampling="uniform")
    out = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, X.to(DEV), ranks, J, sweeps, seed, T.TR_PREC_FP64, out,
                     init_cores=[to_dev_core(c) for c in init])
    for k in range(len(dims)):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8


def test_uniform_mixed_end_to_end(ctx):
    dims, ranks, J, sweeps = (40, 36, 32), (5, 5, 5), 1500, 6
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=3, rel_noise=0.05)
    init = np_cores(dims, ranks, 4)
    ref = orc.tr_als_sampled(X.double().numpy(), init, J, sweeps, 5, sampling="uniform")
    e_ref = orc.rel_error(ref, X.double().numpy())
    Xd = X.to(DEV)
    out = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, 5, T.TR_PREC_MIXED, out,
                     init_cores=[to_dev_core(c) for c in init])
    e_gpu = T.tr_rel_error(ctx, Xd, ranks, out)
    assert abs(e_gpu - e_ref) < 0.01 * e_ref


def test_uniform_batched_matches_oracle_fp64(ctx):
    shapes = [((30, 25, 20), (3, 4, 2), 200), ((12, 9, 10, 11), (2, 3, 2, 3), 150),
              ((40, 6, 33), (4, 3, 5), 250), ((21, 17), (3, 5), 100)]
    probs = []
    for i, (d, r, J) in enumerate(shapes):
        X, _ = inputs.tr_plus_noise(d, r, seed=11 + i, rel_noise=1e-2, dtype=torch.float64)
        init = np_cores(d, r, 1011 + i)
        probs.append(dict(X=X.to(DEV), Xh=X, ranks=r, J=J, seed=18 + i, init=True,
                          cores=[to_dev_core(c) for c in init], init_np=init))
    sweeps = 2
    T.tr_als_sampled_batched(ctx, probs, sweeps, T.TR_PREC_FP64)
    for pr in probs:
        ref = orc.tr_als_sampled(pr["Xh"].numpy(), pr["init_np"], pr["J"], sweeps, pr["seed"],
                                 solver="normal", sampling="uniform")
        for k in range(len(ref)):
            assert rel(to_paper(pr["cores"][k]), ref[k]) < 1e-8


def test_sampling_switch(ctx):
    assert T.tr_get_sampling(ctx) == T.TR_SAMPLING_UNIFORM
    with pytest.raises(T.TrError) as e:
        T.tr_set_sampling(ctx, 2)
    assert e.value.status == T.TR_ERR_INVALID_ARG
    assert T.tr_get_sampling(ctx) == T.TR_SAMPLING_UNIFORM
    dims, ranks, J = (30, 25, 20), (3, 4, 2), 300
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=8, rel_noise=1e-2)
    Xd = X.to(DEV)
    init = [to_dev_core(c) for c in np_cores(dims, ranks, 9)]

    def run(sampling):
        T.tr_set_sampling(ctx, sampling)
        out = T.empty_cores(dims, ranks)
        T.tr_als_sampled(ctx, Xd, ranks, J, 2, 4, T.TR_PREC_MIXED, out, init_cores=init)
        return [c.clone() for c in out]

    lev = run(T.TR_SAMPLING_LEVERAGE)
    uni = run(T.TR_SAMPLING_UNIFORM)
    lev2 = run(T.TR_SAMPLING_LEVERAGE)
    assert all(torch.equal(a, b) for a, b in zip(lev, lev2))
    assert not all(torch.equal(a, b) for a, b in zip(lev, uni))
