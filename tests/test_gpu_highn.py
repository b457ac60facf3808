"""The high-order shape of Sec. 5 (10-way 4 x ... x 4 tensors, TR ranks 10): every mode is
wide (I = 4 < L = 100). On the oscillatory function tensors the fast modes' cores become
numerically rank-deficient (singular-value ratios down to 1e-12), so their distributions
depend on resolving singular values far below sqrt(eps); the library takes them by
one-sided Jacobi with the singular-value rank rule. Whole FP64 driver sweeps on the three
oscillatory tensors therefore match the oracle (same draws, cores within 1e-8), and so does
each stage of an update. The mixed path's final error is compared where its LS steps stay
within FP32 resolution (kappa(M) * eps32 < 1; the Airy tensor and a TR + noise tensor)."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
DIMS, RANKS = (4,) * 10, (10,) * 10


@pytest.fixture(scope="module")
def ctx():
    c = T.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_dev_core(core_paper):
    return torch.from_numpy(np.ascontiguousarray(np.transpose(core_paper, (1, 0, 2)))).to(DEV)


def to_paper(core_dev):
    return np.ascontiguousarray(np.transpose(core_dev.cpu().numpy(), (1, 0, 2)))


def test_highn_core_update_stages_match_oracle(ctx):
    """One update per mode position at N = 10, stage by stage: draws bit-exact, design rows,
    fibres and the FP64 solve against the oracle's, from the oracle's distributions."""
    X = inputs.oscillatory("linear_growth", dtype=torch.float64)
    Xn = X.numpy()
    Xd = X.to(DEV)
    cores = [c.numpy() for c in inputs.random_cores(DIMS, RANKS, 17)]
    ps, cdfs = zip(*[orc.core_distribution(c) for c in cores])
    dev_cores = [to_dev_core(c) for c in cores]
    pd = [torch.from_numpy(p).to(DEV) for p in ps]
    cd = [torch.from_numpy(c).to(DEV) for c in cdfs]
    J = 1500
    for n in (0, 4, 9):
        idx_o, w_o = orc.draw_samples(list(ps), list(cdfs), n, J, 3, n)
        idx = torch.empty((J, 9), dtype=torch.int32, device=DEV)
        w = torch.empty(J, dtype=torch.float64, device=DEV)
        T.tr_sample(ctx, n, DIMS, pd, cd, J, 3, n, idx, w)
        T.tr_status_sync(ctx)
        np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
        np.testing.assert_allclose(w.cpu().numpy(), w_o, rtol=1e-14)
        A = torch.empty((J, 100), dtype=torch.float64, device=DEV)
        T.tr_subchain(ctx, n, DIMS, RANKS, dev_cores, idx, w, A)
        A_o = orc.sampled_subchain(cores, n, idx_o, w_o)
        assert rel(A.cpu().numpy(), A_o) < 1e-12
        Y = torch.empty((J, 4), dtype=torch.float64, device=DEV)
        T.tr_gather(ctx, Xd, n, idx, w, Y)
        Y_o = orc.sampled_fibres(Xn, n, idx_o, w_o)
        assert rel(Y.cpu().numpy(), Y_o) < 1e-14
        out = torch.empty((4, 10, 10), dtype=torch.float64, device=DEV)
        T.tr_solve(ctx, A, Y, 10, 10, T.TR_PREC_FP64, out)
        T.tr_status_sync(ctx)
        ref = orc.core_from_solution(orc.sampled_ls_normal(A_o, Y_o), 10, 10)
        assert rel(to_paper(out), ref) < 1e-9


@pytest.mark.parametrize("name", ["linear_growth", "airy", "chirp"])
def test_highn_sweeps_match_oracle_fp64(ctx, name):
    """Two whole FP64 sweeps of the driver (fused sampler, distributions of the wide cores by
    Jacobi) on the oscillatory tensor itself: every core within 1e-8 of the oracle's. One
    different draw would move a core by far more (about 1e-3)."""
    X = inputs.oscillatory(name, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(DIMS, RANKS, 7)]
    J = 1500
    ref = orc.tr_als_sampled(X.numpy(), init, J, 2, 3, solver="normal")
    out = T.empty_cores(DIMS, RANKS)
    T.tr_als_sampled(ctx, X.to(DEV), RANKS, J, 2, 3, T.TR_PREC_FP64, out,
                     init_cores=[to_dev_core(c) for c in init])
    for k in range(10):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8, k


def test_highn_sweep_matches_oracle_fp64_tr_noise(ctx):
    """A whole FP64 sweep on a 10-way TR + noise tensor of the same shape and ranks."""
    X, _ = inputs.tr_plus_noise(DIMS, RANKS, seed=6, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(DIMS, RANKS, 7)]
    J = 1500
    ref = orc.tr_als_sampled(X.numpy(), init, J, 1, 3, solver="normal")
    out = T.empty_cores(DIMS, RANKS)
    T.tr_als_sampled(ctx, X.to(DEV), RANKS, J, 1, 3, T.TR_PREC_FP64, out,
                     init_cores=[to_dev_core(c) for c in init])
    for k in range(10):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8


def test_highn_wide_leverage_of_rank_deficient_cores(ctx):
    """tr_leverage on the cores one oracle sweep leaves on the linear-growth tensor (4 x 100
    unfoldings with singular-value ratios down to about 1e-12): p and the CDF equal the
    oracle's SVD-based distribution."""
    X = inputs.oscillatory("linear_growth", dtype=torch.float64).numpy()
    init = [c.numpy() for c in inputs.random_cores(DIMS, RANKS, 7)]
    cores = orc.tr_als_sampled(X, init, 1500, 1, 3, solver="normal")
    ratios = []
    for c in cores:
        sv = np.linalg.svd(orc.core_unfold2(c), compute_uv=False)
        ratios.append(sv[-1] / sv[0])
        p_o, cdf_o = orc.core_distribution(c)
        p = torch.empty(4, dtype=torch.float64, device=DEV)
        cdf = torch.empty(4, dtype=torch.float64, device=DEV)
        T.tr_leverage(ctx, to_dev_core(c), p, cdf)
        T.tr_status_sync(ctx)
        np.testing.assert_allclose(p.cpu().numpy(), p_o, rtol=0, atol=1e-14)
        np.testing.assert_allclose(cdf.cpu().numpy(), cdf_o, rtol=0, atol=1e-14)
    assert min(ratios) < 1e-9   # the case the Gram-based route cannot resolve


def test_highn_mixed_final_error(ctx):
    X, _ = inputs.tr_plus_noise(DIMS, RANKS, seed=12, rel_noise=1e-2)
    init = [c.numpy() for c in inputs.random_cores(DIMS, RANKS, 23)]
    J, sweeps = 2000, 3
    ref = orc.tr_als_sampled(X.double().numpy(), init, J, sweeps, 4)
    e_ref = orc.rel_error(ref, X.double().numpy())
    Xd = X.to(DEV)
    out = T.empty_cores(DIMS, RANKS)
    T.tr_als_sampled(ctx, Xd, RANKS, J, sweeps, 4, T.TR_PREC_MIXED, out,
                     init_cores=[to_dev_core(c) for c in init])
    e_gpu = T.tr_rel_error(ctx, Xd, RANKS, out)
    assert abs(e_gpu - e_ref) < 0.01 * e_ref


def test_highn_mixed_final_error_airy(ctx):
    """The mixed path on an oscillatory tensor whose LS steps it can resolve (Airy: kappa(M)
    up to about 2e7 along the trajectory): final error within 1% of the oracle's."""
    X = inputs.oscillatory("airy", dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(DIMS, RANKS, 7)]
    ref = orc.tr_als_sampled(X.numpy(), init, 2000, 3, 4)
    e_ref = orc.rel_error(ref, X.numpy())
    Xf = X.float().to(DEV)
    out = T.empty_cores(DIMS, RANKS)
    T.tr_als_sampled(ctx, Xf, RANKS, 2000, 3, 4, T.TR_PREC_MIXED, out,
                     init_cores=[to_dev_core(c) for c in init])
    e_gpu = T.tr_rel_error(ctx, Xf, RANKS, out)
    assert abs(e_gpu - e_ref) < 0.01 * e_ref
