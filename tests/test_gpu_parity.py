"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, stage by stage and
end to end. Tolerances: sampled indices bit-exact; FP64 path <= 1e-10 relative Frobenius
per core update; mixed path <= 1e-4; end-to-end final relative error within 1 % of the
oracle's."""

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


def np_cores(dims, ranks, seed):
    return [c.numpy() for c in inputs.random_cores(dims, ranks, seed)]


# ----------------------------------------------------------------------------------------
# a2: sampler
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("dims,n,J", [((7, 300, 5), 0, 1), ((50, 40, 30), 1, 4001),
                                      ((3, 4, 5, 6, 7), 2, 1000), ((200, 2), 0, 777),
                                      ((500, 500, 500), 2, 4000)])
def test_sample_bit_exact(ctx, dims, n, J):
    N = len(dims)
    ps = [inputs.random_distribution(d, seed=10 + k, zero_frac=0.3).numpy() for k, d in
          enumerate(dims)]
    cdfs = [np.cumsum(p) for p in ps]
    seed, uid = 12345678901, 2 ** 33 + 5
    idx_o, w_o = orc.draw_samples(ps, cdfs, n, J, seed, uid)
    pd = [torch.from_numpy(p).to(DEV) for p in ps]
    cd = [torch.from_numpy(c).to(DEV) for c in cdfs]
    idx = torch.empty((J, N - 1), dtype=torch.int32, device=DEV)
    w = torch.empty(J, dtype=torch.float64, device=DEV)
    T.tr_sample(ctx, n, dims, pd, cd, J, seed, uid, idx, w)
    T.tr_status_sync(ctx)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    np.testing.assert_array_equal(w.cpu().numpy(), w_o)


def test_sample_rounding_overflow_goes_to_last_positive(ctx):
    """cdf[last] < 1: uniforms above it take the largest index with positive mass."""
    p = np.array([0.3, 0.0, 0.3, 0.3, 0.0, 0.0])
    cdf = np.cumsum(p)                                  # ends at 0.9
    q = np.full(4, 0.25)
    ps, cdfs = [q, p], [np.cumsum(q), cdf]
    J = 5000
    idx_o, w_o = orc.draw_samples(ps, cdfs, 0, J, 7, 1)
    assert np.any(idx_o[:, 0] == 3)
    idx = torch.empty((J, 1), dtype=torch.int32, device=DEV)
    w = torch.empty(J, dtype=torch.float64, device=DEV)
    T.tr_sample(ctx, 0, (4, 6), [torch.from_numpy(x).to(DEV) for x in ps],
                [torch.from_numpy(x).to(DEV) for x in cdfs], J, 7, 1, idx, w)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    np.testing.assert_array_equal(w.cpu().numpy(), w_o)


# ----------------------------------------------------------------------------------------
# a1: leverage distribution
# ----------------------------------------------------------------------------------------
def _leverage_gpu(ctx, core_paper):
    Rl, I, Rr = core_paper.shape
    p = torch.empty(I, dtype=torch.float64, device=DEV)
    c = torch.empty(I, dtype=torch.float64, device=DEV)
    T.tr_leverage(ctx, to_dev_core(core_paper), p, c)
    return p, c


@pytest.mark.parametrize("I,Rl,Rr", [(500, 10, 10), (1, 2, 3), (3, 10, 10), (37, 4, 5),
                                     (1000, 16, 16), (20, 4, 5), (19, 4, 5), (2000, 10, 10),
                                     (129, 1, 1)])
def test_leverage_matches_oracle(ctx, I, Rl, Rr):
    core = np.random.default_rng(I * 7 + Rl).standard_normal((Rl, I, Rr))
    p_o, c_o = orc.core_distribution(core)
    p, c = _leverage_gpu(ctx, core)
    T.tr_status_sync(ctx)
    np.testing.assert_allclose(p.cpu().numpy(), p_o, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(c.cpu().numpy(), c_o, rtol=0, atol=1e-12)


def test_leverage_rank_deficient(ctx):
    rng = np.random.default_rng(3)
    Rl, I, Rr = 4, 60, 5
    u = rng.standard_normal((Rl, I))
    v = rng.standard_normal(Rr)
    core = u[:, :, None] * v[None, None, :]              # G_(2) has rank Rl = 4
    p_o, _ = orc.core_distribution(core)
    p, _ = _leverage_gpu(ctx, core)
    T.tr_status_sync(ctx)
    np.testing.assert_allclose(p.cpu().numpy(), p_o, rtol=1e-8, atol=1e-13)


def test_leverage_zero_core_is_singular(ctx):
    core = np.zeros((3, 10, 3))
    p, c = _leverage_gpu(ctx, core)
    with pytest.raises(T.TrError) as e:
        T.tr_status_sync(ctx)
    assert e.value.status == T.TR_ERR_SINGULAR
    np.testing.assert_allclose(p.cpu().numpy(), 0.1)


# ----------------------------------------------------------------------------------------
# a3: subchain, a4: gather
# ----------------------------------------------------------------------------------------
CHAIN_CASES = [((6, 7, 8), (3, 4, 2)), ((9, 5, 7, 4), (2, 3, 4, 5)), ((4, 3, 5, 2, 6), (2, 2, 3, 2, 4)),
               ((11, 13), (3, 5)), ((30, 30, 30), (16, 16, 16))]


@pytest.mark.parametrize("dims,ranks", CHAIN_CASES)
@pytest.mark.parametrize("f64", [True, False])
def test_subchain_matches_oracle(ctx, dims, ranks, f64):
    N = len(dims)
    cores = np_cores(dims, ranks, 21)
    rng = np.random.default_rng(22)
    J = 333
    for n in range(N):
        others = orc.ring_modes(N, n)
        idx = np.stack([rng.integers(0, dims[m], J) for m in others], axis=1)
        w = rng.uniform(0.1, 3.0, J)
        ref = orc.sampled_subchain(cores, n, idx, w)
        L = ref.shape[1]
        A = torch.empty((J, L), dtype=torch.float64 if f64 else torch.float32, device=DEV)
        T.tr_subchain(ctx, n, dims, ranks, [to_dev_core(c) for c in cores],
                      torch.from_numpy(idx.astype(np.int32)).to(DEV),
                      torch.from_numpy(w).to(DEV), A)
        T.tr_status_sync(ctx)
        assert rel(A.cpu().numpy(), ref) < (1e-13 if f64 else 2e-6)


def test_subchain_rejects_out_of_range_index(ctx):
    dims, ranks = (6, 7, 8), (3, 4, 2)
    cores = [to_dev_core(c) for c in np_cores(dims, ranks, 1)]
    idx = torch.tensor([[1, 2], [9, 0], [3, 3]], dtype=torch.int32, device=DEV)
    A = torch.full((3, 6), 7.0, dtype=torch.float64, device=DEV)
    T.tr_subchain(ctx, 0, dims, ranks, cores, idx, None, A)
    with pytest.raises(T.TrError) as e:
        T.tr_status_sync(ctx)
    assert e.value.status == T.TR_ERR_INVALID_ARG
    assert torch.all(A[1] == 0)


@pytest.mark.parametrize("dims", [(13, 17, 19), (5, 6, 7, 8), (40, 3), (2, 3, 4, 5, 6),
                                  (300, 7, 5), (2, 600, 3)])
@pytest.mark.parametrize("xdt,ydt", [(torch.float64, torch.float64), (torch.float32, torch.float32),
                                     (torch.float32, torch.float64)])
def test_gather_matches_oracle(ctx, dims, xdt, ydt):
    N = len(dims)
    X = torch.randn(dims, generator=torch.Generator().manual_seed(5), dtype=torch.float64).to(xdt)
    Xn = X.double().numpy()
    Xd = X.to(DEV)
    rng = np.random.default_rng(6)
    J = 257
    for n in range(N):
        others = orc.ring_modes(N, n)
        idx = np.stack([rng.integers(0, dims[m], J) for m in others], axis=1)
        w = rng.uniform(0.1, 3.0, J)
        ref = orc.sampled_fibres(Xn, n, idx, w)
        Y = torch.empty((J, dims[n]), dtype=ydt, device=DEV)
        T.tr_gather(ctx, Xd, n, torch.from_numpy(idx.astype(np.int32)).to(DEV),
                    torch.from_numpy(w).to(DEV), Y)
        T.tr_status_sync(ctx)
        tol = 0.0 if ydt == torch.float64 else 1.2e-7
        np.testing.assert_allclose(Y.cpu().double().numpy(), ref, rtol=tol, atol=0)


# ----------------------------------------------------------------------------------------
# a5 + a6: normal equations, Cholesky, refinement
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("J,Rl,Rr,I", [(100, 10, 10, 500), (4000, 10, 10, 500), (2000, 5, 5, 100),
                                       (300, 16, 16, 77), (1, 1, 1, 3), (50, 3, 2, 1)])
def test_solve_fp64(ctx, J, Rl, Rr, I):
    rng = np.random.default_rng(J + I)
    L = Rl * Rr
    A = rng.standard_normal((J, L))
    Y = A @ rng.standard_normal((L, I)) + 0.1 * rng.standard_normal((J, I))
    Z = orc.sampled_ls_normal(A, Y)
    ref = orc.core_from_solution(Z, Rl, Rr)
    out = torch.empty((I, Rl, Rr), dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, torch.from_numpy(A).to(DEV), torch.from_numpy(Y).to(DEV), Rl, Rr,
               T.TR_PREC_FP64, out)
    T.tr_status_sync(ctx)
    assert rel(to_paper(out), ref) < 1e-10


@pytest.mark.parametrize("J,Rl,Rr,I", [(4000, 10, 10, 500), (8000, 10, 10, 2000), (300, 16, 16, 77)])
def test_solve_mixed(ctx, J, Rl, Rr, I):
    rng = np.random.default_rng(J + 1)
    L = Rl * Rr
    A = rng.standard_normal((J, L)).astype(np.float32)
    Y = (A.astype(np.float64) @ rng.standard_normal((L, I)) +
         0.05 * rng.standard_normal((J, I))).astype(np.float32)
    Z = orc.sampled_ls_normal(A.astype(np.float64), Y.astype(np.float64))
    ref = orc.core_from_solution(Z, Rl, Rr)
    out = torch.empty((I, Rl, Rr), dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, torch.from_numpy(A).to(DEV), torch.from_numpy(Y).to(DEV), Rl, Rr,
               T.TR_PREC_MIXED, out)
    T.tr_status_sync(ctx)
    assert rel(to_paper(out), ref) < 1e-4


def test_solve_mixed_column_scaled_takes_the_fp64_factor(ctx):
    """Columns scaled down to 10^-3.5: the FP32 factorisation of the mixed LS step meets a
    pivot below n*eps32*max diag, so the step factors in FP64 instead (an FP32-only step
    would report the matrix singular). Cholesky's accuracy depends on the column-equilibrated
    matrix, so the result still matches the oracle."""
    J, Rl, Rr, I = 2000, 4, 4, 60
    rng = np.random.default_rng(77)
    L = Rl * Rr
    scale = 10.0 ** (-3.5 * np.arange(L) / (L - 1))
    A = (rng.standard_normal((J, L)) * scale).astype(np.float32)
    Y = (A.astype(np.float64) @ rng.standard_normal((L, I)) +
         0.05 * rng.standard_normal((J, I))).astype(np.float32)
    Z = orc.sampled_ls_normal(A.astype(np.float64), Y.astype(np.float64))
    M = A.astype(np.float64).T @ A.astype(np.float64)
    piv = np.diag(np.linalg.cholesky(M)) ** 2
    assert piv.min() < L * 2.0 ** -23 * np.diag(M).max()      # the FP32 branch must stop
    ref = orc.core_from_solution(Z, Rl, Rr)
    out = torch.empty((I, Rl, Rr), dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, torch.from_numpy(A).to(DEV), torch.from_numpy(Y).to(DEV), Rl, Rr,
               T.TR_PREC_MIXED, out)
    T.tr_status_sync(ctx)
    assert rel(to_paper(out), ref) < 1e-4


def test_solve_mixed_singular_leaves_core_unchanged(ctx):
    J, Rl, Rr, I = 5, 4, 4, 9                 # J < L: the normal matrix is singular
    A = torch.randn((J, Rl * Rr), dtype=torch.float32, device=DEV)
    Y = torch.randn((J, I), dtype=torch.float32, device=DEV)
    out = torch.full((I, Rl, Rr), 3.0, dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, A, Y, Rl, Rr, T.TR_PREC_MIXED, out)
    with pytest.raises(T.TrError) as e:
        T.tr_status_sync(ctx)
    assert e.value.status == T.TR_ERR_SINGULAR
    assert torch.all(out == 3.0)


def test_solve_singular_leaves_core_unchanged(ctx):
    J, Rl, Rr, I = 5, 4, 4, 9                 # J < L: the normal matrix is singular
    A = torch.randn((J, Rl * Rr), dtype=torch.float64, device=DEV)
    Y = torch.randn((J, I), dtype=torch.float64, device=DEV)
    out = torch.full((I, Rl, Rr), 3.0, dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, A, Y, Rl, Rr, T.TR_PREC_FP64, out)
    with pytest.raises(T.TrError) as e:
        T.tr_status_sync(ctx)
    assert e.value.status == T.TR_ERR_SINGULAR
    assert torch.all(out == 3.0)


def test_invalid_arguments_are_rejected_before_launch(ctx):
    out = torch.empty((3, 2, 2), dtype=torch.float64, device=DEV)
    A = torch.randn((8, 4), dtype=torch.float32, device=DEV)
    Y = torch.randn((8, 3), dtype=torch.float32, device=DEV)
    with pytest.raises(T.TrError) as e:
        T.tr_solve(ctx, A, Y, 2, 2, T.TR_PREC_FP64, out)      # FP64 path needs FP64 inputs
    assert e.value.status == T.TR_ERR_INVALID_ARG
    X = torch.randn((4, 5, 6), device=DEV)
    cores = T.empty_cores((4, 5, 6), (2, 2, 2))
    with pytest.raises(T.TrError) as e:
        T.tr_als_sampled(ctx, X, (2, 17, 2), 10, 1, 0, T.TR_PREC_MIXED, cores)
    assert e.value.status == T.TR_ERR_INVALID_ARG
    with pytest.raises(T.TrError) as e:
        T.tr_als_sampled(ctx, X, (2, 2, 2), 0, 1, 0, T.TR_PREC_MIXED, cores)
    assert e.value.status == T.TR_ERR_INVALID_ARG


# ----------------------------------------------------------------------------------------
# One whole core update (a2-a6) given the same prior cores and distributions
# ----------------------------------------------------------------------------------------
def _gpu_update(ctx, X_dev, cores_paper, ps, cdfs, n, J, seed, uid, prec):
    dims = list(X_dev.shape)
    N = len(dims)
    ranks = [c.shape[2] for c in cores_paper]
    f64 = prec == T.TR_PREC_FP64
    dt = torch.float64 if f64 else torch.float32
    dev_cores = [to_dev_core(c) for c in cores_paper]
    pd = [torch.from_numpy(p).to(DEV) if p is not None else None for p in ps]
    cd = [torch.from_numpy(c).to(DEV) if c is not None else None for c in cdfs]
    idx = torch.empty((J, N - 1), dtype=torch.int32, device=DEV)
    w = torch.empty(J, dtype=torch.float64, device=DEV)
    T.tr_sample(ctx, n, dims, pd, cd, J, seed, uid, idx, w)
    Rl, _, Rr = cores_paper[n].shape
    A = torch.empty((J, Rl * Rr), dtype=dt, device=DEV)
    Y = torch.empty((J, dims[n]), dtype=dt, device=DEV)
    T.tr_subchain(ctx, n, dims, ranks, dev_cores, idx, w, A)
    T.tr_gather(ctx, X_dev, n, idx, w, Y)
    out = torch.empty((dims[n], Rl, Rr), dtype=torch.float64, device=DEV)
    T.tr_solve(ctx, A, Y, Rl, Rr, prec, out)
    T.tr_status_sync(ctx)
    return to_paper(out), idx.cpu().numpy()


@pytest.mark.parametrize("dims,ranks,J,prec", [
    ((60, 50, 40), (4, 5, 3), 500, T.TR_PREC_FP64),
    ((60, 50, 40), (4, 5, 3), 500, T.TR_PREC_MIXED),
    ((20, 15, 10, 12), (3, 4, 2, 3), 400, T.TR_PREC_FP64),
    ((20, 15, 10, 12), (3, 4, 2, 3), 400, T.TR_PREC_MIXED),
    ((100, 100, 100), (5, 5, 5), 2000, T.TR_PREC_FP64),
])
def test_core_update_matches_oracle(ctx, dims, ranks, J, prec):
    xdt = torch.float64 if prec == T.TR_PREC_FP64 else torch.float32
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=3, rel_noise=1e-2, dtype=xdt)
    Xn = X.double().numpy()
    cores = np_cores(dims, ranks, 4)
    N = len(dims)
    ps, cdfs = [None] * N, [None] * N
    for k in range(N):
        ps[k], cdfs[k] = orc.core_distribution(cores[k])
    for n in range(N):
        ref, idx_o, _ = orc.sampled_core_update(Xn, cores, ps, cdfs, n, J, 99, 1000 + n,
                                                 solver="normal")
        got, idx_g = _gpu_update(ctx, X.to(DEV), cores, ps, cdfs, n, J, 99, 1000 + n, prec)
        np.testing.assert_array_equal(idx_g, idx_o)
        assert rel(got, ref) < (1e-10 if prec == T.TR_PREC_FP64 else 1e-4)


def test_core_update_full_size_mixed(ctx):
    """The 500^3, rank-10, J = 4000 workload the benchmark times: one update per mode, the
    sampler bit-exact and the new core within 1e-4 of the oracle."""
    wl = inputs.WORKLOADS["tr3_500_r10_fp32"]
    X, _ = inputs.tr_plus_noise(wl["dims"], wl["ranks"], seed=wl["seed"],
                                rel_noise=wl["rel_noise"], device=DEV, dtype=torch.float32)
    Xn = X.cpu().numpy()
    cores = np_cores(wl["dims"], wl["ranks"], wl["init_seed"])
    N = 3
    ps, cdfs = [None] * N, [None] * N
    for k in range(N):
        ps[k], cdfs[k] = orc.core_distribution(cores[k])
    for n in range(N):
        ref, idx_o, _ = orc.sampled_core_update(Xn, cores, ps, cdfs, n, wl["J"], wl["sample_seed"],
                                                 n, solver="normal")
        got, idx_g = _gpu_update(ctx, X, cores, ps, cdfs, n, wl["J"], wl["sample_seed"], n,
                                 T.TR_PREC_MIXED)
        np.testing.assert_array_equal(idx_g, idx_o)
        assert rel(got, ref) < 1e-4


# ----------------------------------------------------------------------------------------
# Fit and the whole method
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("dims,ranks,xdt", [((30, 20, 25), (3, 4, 5), torch.float64),
                                            ((30, 20, 25), (3, 4, 5), torch.float32),
                                            ((6, 5, 7, 4), (2, 3, 2, 4), torch.float64),
                                            ((50, 40), (4, 6), torch.float64),
                                            # mode splits s = 2 (cols 300, 16-byte rows)
                                            # and s = 2 of 5 modes, FP32
                                            ((20, 30, 300), (4, 5, 3), torch.float32),
                                            ((8, 6, 7, 5, 9), (3, 2, 4, 3, 2), torch.float32),
                                            ((9, 70, 11, 13), (5, 4, 6, 3), torch.float32),
                                            # K = 110 (tensor cores), K = 144 (SIMT)
                                            ((60, 50, 140), (10, 11, 10), torch.float32),
                                            ((40, 30, 20), (12, 12, 12), torch.float32)])
def test_rel_error_matches_oracle(ctx, dims, ranks, xdt):
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=8, rel_noise=0.05, dtype=xdt)
    cores = np_cores(dims, ranks, 9)
    ref = orc.rel_error(cores, X.double().numpy())
    got = T.tr_rel_error(ctx, X.to(DEV), ranks, [to_dev_core(c) for c in cores])
    assert abs(got - ref) <= (1e-12 if xdt == torch.float64 else 1e-6) * ref


def test_als_sampled_end_to_end_fp64(ctx):
    """The 100^3 rank-5 FP64 workload, J = 2000, 10 sweeps, from the same initial cores."""
    wl = inputs.WORKLOADS["tr3_100_r5_fp64"]
    X, _ = inputs.tr_plus_noise(wl["dims"], wl["ranks"], seed=wl["seed"],
                                rel_noise=wl["rel_noise"], dtype=torch.float64)
    init = np_cores(wl["dims"], wl["ranks"], wl["init_seed"] + 100)
    ref_cores = orc.tr_als_sampled(X.numpy(), init, wl["J"], wl["sweeps"], wl["sample_seed"])
    e_ref = orc.rel_error(ref_cores, X.numpy())
    Xd = X.to(DEV)
    out = T.empty_cores(wl["dims"], wl["ranks"])
    T.tr_als_sampled(ctx, Xd, wl["ranks"], wl["J"], wl["sweeps"], wl["sample_seed"],
                     T.TR_PREC_FP64, out, init_cores=[to_dev_core(c) for c in init])
    e_gpu = T.tr_rel_error(ctx, Xd, wl["ranks"], out)
    e_gpu_oracle = orc.rel_error([to_paper(c) for c in out], X.numpy())
    assert abs(e_gpu - e_gpu_oracle) < 1e-10 * e_gpu_oracle
    assert abs(e_gpu - e_ref) < 0.01 * e_ref


def test_als_sampled_end_to_end_mixed(ctx):
    dims, ranks, J, sweeps = (120, 110, 100), (6, 6, 6), 1000, 8
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=12, rel_noise=1e-2, dtype=torch.float32)
    init = np_cores(dims, ranks, 13)
    ref_cores = orc.tr_als_sampled(X.double().numpy(), init, J, sweeps, 5)
    e_ref = orc.rel_error(ref_cores, X.double().numpy())
    Xd = X.to(DEV)
    out = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, 5, T.TR_PREC_MIXED, out,
                     init_cores=[to_dev_core(c) for c in init])
    e_gpu = T.tr_rel_error(ctx, Xd, ranks, out)
    assert abs(e_gpu - e_ref) < 0.01 * e_ref


def test_als_sampled_is_deterministic_and_host_api_agrees(ctx):
    dims, ranks, J, sweeps = (40, 30, 20), (3, 3, 4), 300, 4
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=2, rel_noise=1e-2, dtype=torch.float32)
    Xd = X.to(DEV)
    a = T.empty_cores(dims, ranks)
    b = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, 77, T.TR_PREC_MIXED, a)
    T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, 77, T.TR_PREC_MIXED, b)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    host = [torch.empty(c.shape, dtype=torch.float64).pin_memory() for c in a]
    T.tr_als_sampled_host(ctx, X.pin_memory(), ranks, J, sweeps, 77, T.TR_PREC_MIXED, host)
    for x, y in zip(a, host):
        assert torch.equal(x.cpu(), y)


@pytest.mark.parametrize("dims,ranks", [((30, 25, 20), (3, 4, 2)), ((12, 9, 10, 11), (2, 3, 2, 3))])
def test_als_sampled_first_sweeps_match_oracle_fp64(ctx, dims, ranks):
    """Two FP64 sweeps of the whole driver (fused sampler + subchain, leverage from B^T on
    the concurrent branch) against the oracle's Alg. 2 with the normal-equation solve: the
    same draws and the same arithmetic up to rounding."""
    J, sweeps, seed = 300, 2, 21
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=6, rel_noise=1e-2, dtype=torch.float64)
    init = np_cores(dims, ranks, 7)
    ref = orc.tr_als_sampled(X.numpy(), init, J, sweeps, seed, solver="normal")
    out = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, X.to(DEV), ranks, J, sweeps, seed, T.TR_PREC_FP64, out,
                     init_cores=[to_dev_core(c) for c in init])
    for k in range(len(dims)):
        assert rel(to_paper(out[k]), ref[k]) < 1e-8


def test_als_sampled_end_to_end_4way_cosine_mixed(ctx):
    """The 4-way smooth workload at reduced size: a sum of 20 separable low-frequency cosine
    products plus 5 % uniform noise, a colour-like mode of size 3 (wide G_(2): I = 3 < L =
    100), TR ranks 10, mixed precision, against the oracle's final fit."""
    dims, ranks, J, sweeps = (48, 40, 3, 300), (10, 10, 10, 10), 3000, 4
    X = inputs.cosine_sum(dims, seed=0)
    init = np_cores(dims, ranks, 31)
    ref = orc.tr_als_sampled(X.double().numpy(), init, J, sweeps, 9)
    e_ref = orc.rel_error(ref, X.double().numpy())
    Xd = X.to(DEV)
    out = T.empty_cores(dims, ranks)
    T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, 9, T.TR_PREC_MIXED, out,
                     init_cores=[to_dev_core(c) for c in init])
    e_gpu = T.tr_rel_error(ctx, Xd, ranks, out)
    assert abs(e_gpu - e_ref) < 0.01 * e_ref
