"""Row a1 as the mixed-precision drivers form it (tr_leverage_planes): the leverage
distribution of a tall matrix held as two FP32 planes, through the FP32-preconditioned
series or, when the preconditioner is too poor, the double-float factorisation with FP64
fallback. Compared with the oracle's SVD-based leverage scores (Def. 4) of the same matrix
(hi + lo in FP64)."""

import os

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = T.Context(0)
    yield c
    c.close()


def planes(A):
    hi = A.astype(np.float32)
    lo = (A - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def with_condition(I, L, kappa, seed):
    """I x L matrix with singular values spread geometrically from 1 to 1/kappa."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((I, L)))
    V, _ = np.linalg.qr(rng.standard_normal((L, L)))
    s = np.geomspace(1.0, 1.0 / kappa, L)
    return (U * s) @ V.T


def run(ctx, hi, lo):
    I, L = hi.shape
    p = torch.empty(I, dtype=torch.float64, device=DEV)
    c = torch.empty(I, dtype=torch.float64, device=DEV)
    br = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    T.tr_leverage_planes(ctx, torch.from_numpy(hi).to(DEV), torch.from_numpy(lo).to(DEV), p, c,
                         br)
    T.tr_status_sync(ctx)
    return p.cpu().numpy(), c.cpu().numpy(), int(br.item())


def oracle_p(hi, lo):
    A = hi.astype(np.float64) + lo.astype(np.float64)
    ell = orc.leverage_scores(A)
    p = ell / ell.sum()
    return p, np.cumsum(p)


@pytest.mark.parametrize("I,L", [(500, 100), (300, 64), (1000, 36), (40, 4), (200, 128),
                                 (4001, 100)])
def test_gaussian_takes_the_preconditioned_form(ctx, I, L):
    A = np.random.default_rng(I + 3 * L).standard_normal((I, L))
    hi, lo = planes(A)
    p, c, br = run(ctx, hi, lo)
    p_o, c_o = oracle_p(hi, lo)
    assert br == 0
    np.testing.assert_allclose(p, p_o, rtol=1e-10, atol=1e-16)
    np.testing.assert_allclose(c, c_o, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kappa", [3.0, 10.0, 30.0])
def test_moderate_condition_takes_the_preconditioned_form(ctx, kappa):
    hi, lo = planes(with_condition(500, 100, kappa, 5))
    p, _, br = run(ctx, hi, lo)
    p_o, _ = oracle_p(hi, lo)
    assert br == 0
    np.testing.assert_allclose(p, p_o, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("kappa", [100.0, 300.0])
def test_either_branch_is_accurate(ctx, kappa):
    """Near the switch (||E||_F about 1e-2): whichever branch runs, p agrees with the
    oracle to the double-float factorisation's accuracy."""
    hi, lo = planes(with_condition(500, 100, kappa, 6))
    p, _, br = run(ctx, hi, lo)
    p_o, _ = oracle_p(hi, lo)
    assert br in (0, 1)
    np.testing.assert_allclose(p, p_o, rtol=1e-8, atol=1e-16)


@pytest.mark.parametrize("I,L", [(129, 128), (128, 128)])
def test_square_gaussian(ctx, I, L):
    """Nearly square Gaussian matrices (condition in the hundreds): either branch, and
    leverage close to 1 in every row."""
    hi, lo = planes(np.random.default_rng(I + L).standard_normal((I, L)))
    p, _, br = run(ctx, hi, lo)
    p_o, _ = oracle_p(hi, lo)
    assert br in (0, 1)
    np.testing.assert_allclose(p, p_o, rtol=1e-7, atol=1e-16)


def test_ill_conditioned_falls_back(ctx):
    hi, lo = planes(with_condition(500, 100, 1e3, 7))
    p, _, br = run(ctx, hi, lo)
    p_o, _ = oracle_p(hi, lo)
    assert br == 1
    np.testing.assert_allclose(p, p_o, rtol=1e-6, atol=1e-16)


def test_dependent_column_falls_back_and_drops_it(ctx):
    A = np.random.default_rng(8).standard_normal((300, 50))
    A[:, 17] = 2.0 * A[:, 3]
    hi, lo = planes(A)
    assert np.array_equal(hi[:, 17].astype(np.float64) + lo[:, 17],
                          2.0 * (hi[:, 3].astype(np.float64) + lo[:, 3]))
    p, _, br = run(ctx, hi, lo)
    p_o, _ = oracle_p(hi, lo)
    assert br == 1
    np.testing.assert_allclose(p, p_o, rtol=1e-8, atol=1e-15)


def test_zero_matrix_is_singular_and_uniform(ctx):
    hi = np.zeros((64, 16), dtype=np.float32)
    I = hi.shape[0]
    p = torch.empty(I, dtype=torch.float64, device=DEV)
    c = torch.empty(I, dtype=torch.float64, device=DEV)
    d = torch.from_numpy(hi).to(DEV)
    T.tr_leverage_planes(ctx, d, d, p, c)
    with pytest.raises(T.TrError) as e:
        T.tr_status_sync(ctx)
    assert e.value.status == T.TR_ERR_SINGULAR
    np.testing.assert_allclose(p.cpu().numpy(), 1.0 / I)


def test_agrees_with_the_factorisation_form(ctx, monkeypatch):
    """The same planes through both branches (the preconditioned form switched off by
    TRALS_LEV_PRECOND=0): equal to the double-float factorisation's accuracy."""
    hi, lo = planes(np.random.default_rng(9).standard_normal((500, 100)))
    p_fast, _, br = run(ctx, hi, lo)
    assert br == 0
    monkeypatch.setenv("TRALS_LEV_PRECOND", "0")
    p_fact, _, br = run(ctx, hi, lo)
    assert br == 1
    np.testing.assert_allclose(p_fast, p_fact, rtol=1e-11, atol=1e-16)


def test_rejects_unsupported_shapes(ctx):
    for I, L in [(50, 100), (300, 3), (300, 129)]:
        z = torch.zeros((I, L), dtype=torch.float32, device=DEV)
        p = torch.empty(I, dtype=torch.float64, device=DEV)
        with pytest.raises(T.TrError) as e:
            T.tr_leverage_planes(ctx, z, z, p, p)
        assert e.value.status == T.TR_ERR_INVALID_ARG


def test_driver_runs_the_fallback_inside_its_graph(ctx, monkeypatch):
    """The mixed driver's graph holds the factorisation fallback as launches gated by a
    device flag. TRALS_LEV_TAU=0 makes every distribution take it; the decomposition must
    then follow the factorisation form (TRALS_LEV_PRECOND=0) draw for draw. A fallback that
    did not run would leave stale distributions and different draws."""
    from paper_2010_08581_gb300 import inputs
    dims, ranks, J, sweeps = (120, 110, 100), (6, 6, 6), 1000, 4
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=12, rel_noise=1e-2, dtype=torch.float32)
    Xd = X.to(DEV)
    init = [inputs.slice_major(c).to(DEV) for c in inputs.random_cores(dims, ranks, 13)]

    def run_driver():
        out = T.empty_cores(dims, ranks)
        T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, 5, T.TR_PREC_MIXED, out, init_cores=init)
        T.tr_status_sync(ctx)
        return [o.cpu().numpy() for o in out], T.tr_rel_error(ctx, Xd, ranks, out)

    fast, e_fast = run_driver()
    monkeypatch.setenv("TRALS_LEV_TAU", "0")
    forced, _ = run_driver()
    monkeypatch.delenv("TRALS_LEV_TAU")
    monkeypatch.setenv("TRALS_LEV_PRECOND", "0")
    fact, e_fact = run_driver()
    for a, b in zip(forced, fact):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)
    assert abs(e_fast - e_fact) <= 0.01 * e_fact
