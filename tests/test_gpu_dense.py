"""Dense TR-ALS (Alg. 1) through the C ABI (tr_als): FP64 sweeps within 1e-8 of the oracle's
Alg. 1 per core (3- and 4-way, ragged sizes, every mode position including the first and the
last), the mixed path's final error within 1 % of the oracle's, the exact-TR case, and the
argument checks."""

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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev_core(core_paper):
    return torch.from_numpy(np.ascontiguousarray(np.transpose(core_paper, (1, 0, 2)))).to(DEV)


def to_paper(core_dev):
    return np.ascontiguousarray(np.transpose(core_dev.cpu().numpy(), (1, 0, 2)))


@pytest.mark.parametrize("dims,ranks,sweeps", [((30, 25, 20), (3, 4, 2), 2),
                                               ((12, 9, 10, 11), (2, 3, 2, 3), 2),
                                               ((40, 6, 33), (4, 3, 5), 1),
                                               ((30, 40), (2, 3), 2)])
def test_dense_sweeps_match_oracle_fp64(ctx, dims, ranks, sweeps):
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=6, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 7)]
    ref = orc.tr_als(X.numpy(), init, sweeps)
    out = T.empty_cores(dims, ranks)
    T.tr_als(ctx, X.to(DEV), ranks, sweeps, 0, T.TR_PREC_FP64, out,
             init_cores=[to_dev_core(c) for c in init])
    for k in range(len(dims)):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8


def test_dense_mixed_matches_oracle_error(ctx):
    dims, ranks, sweeps = (60, 50, 40), (5, 5, 5), 6
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=3, rel_noise=0.02)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 4)]
    e_ref = orc.rel_error(orc.tr_als(X.double().numpy(), init, sweeps), X.double().numpy())
    Xd = X.to(DEV)
    out = T.empty_cores(dims, ranks)
    T.tr_als(ctx, Xd, ranks, sweeps, 0, T.TR_PREC_MIXED, out,
             init_cores=[to_dev_core(c) for c in init])
    e_gpu = T.tr_rel_error(ctx, Xd, ranks, out)
    assert abs(e_gpu - e_ref) < 0.01 * e_ref


def test_dense_fp64_x_on_the_mixed_path(ctx):
    """X in FP64 with the mixed LS step: the unfolding converts it to FP32 rows."""
    dims, ranks = (20, 18, 16), (3, 3, 3)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=8, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 9)]
    ref = orc.tr_als(X.numpy(), init, 2)
    out = T.empty_cores(dims, ranks)
    T.tr_als(ctx, X.to(DEV), ranks, 2, 0, T.TR_PREC_MIXED, out,
             init_cores=[to_dev_core(c) for c in init])
    for k in range(3):
        assert rel(to_paper(out[k]), ref[k]) < 1e-4


def test_dense_recovers_exact_tr(ctx):
    """Noise-free TR from the start at which the oracle's Alg. 1 converges (oracle pin)."""
    rng = np.random.default_rng(0)
    dims, ranks = (6, 7, 8), (2, 2, 2)
    N = 3
    true = [rng.standard_normal((ranks[(k - 1) % N], dims[k], ranks[k])) for k in range(N)]
    init = [rng.standard_normal((ranks[(k - 1) % N], dims[k], ranks[k])) for k in range(N)]
    X = torch.from_numpy(np.ascontiguousarray(orc.tr_reconstruct(true))).to(DEV)
    out = T.empty_cores(dims, ranks)
    T.tr_als(ctx, X, ranks, 300, 0, T.TR_PREC_FP64, out,
             init_cores=[to_dev_core(c) for c in init])
    assert T.tr_rel_error(ctx, X, ranks, out) < 1e-9


def test_dense_rejects_bad_arguments(ctx):
    X = torch.zeros((4, 5, 6), dtype=torch.float32, device=DEV)
    out = T.empty_cores((4, 5, 6), (2, 2, 2))
    with pytest.raises(T.TrError) as e:
        T.tr_als(ctx, X, (2, 2, 2), -1, 0, T.TR_PREC_MIXED, out)
    assert e.value.status == T.TR_ERR_INVALID_ARG
    with pytest.raises(T.TrError) as e:
        T.tr_als(ctx, X, (2, 17, 2), 1, 0, T.TR_PREC_MIXED, out)
    assert e.value.status == T.TR_ERR_INVALID_ARG
