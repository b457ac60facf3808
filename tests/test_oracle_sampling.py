"""Pins for the oracle's random numbers, leverage scores and sampler (Def. 4, Def. 5,
eq. for p^(n), eq. for q^{!=n}, Alg. 3, Lemma 6). CPU only."""

import itertools
import os

import numpy as np
import pytest
from scipy import stats

import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = orc.philox4x32_10(np.array(v[:4], dtype=np.uint64), v[4:6])
        assert [int(x) for x in out] == v[6:]
        n += 1
    assert n == 3


def test_philox_uniforms_are_uniform():
    u0 = orc.philox_uniforms(200000, 0, seed=123, update_id=5)
    u1 = orc.philox_uniforms(200000, 1, seed=123, update_id=5)
    u2 = orc.philox_uniforms(200000, 2, seed=123, update_id=5)
    for u in (u0, u1, u2):
        assert u.min() >= 0.0 and u.max() < 1.0
        counts = np.histogram(u, bins=20, range=(0, 1))[0]
        assert stats.chisquare(counts).pvalue > 1e-4
    assert abs(np.corrcoef(u0, u1)[0, 1]) < 0.01
    assert abs(np.corrcoef(u0, u2)[0, 1]) < 0.01
    # different update ids give different streams
    assert not np.array_equal(u0, orc.philox_uniforms(200000, 0, seed=123, update_id=6))
    # 53-bit resolution: all values are multiples of 2^-53
    assert np.all(np.floor(u0 * 2.0 ** 53) == u0 * 2.0 ** 53)


def _hat_diag_qr(A):
    """Leverage scores through Householder QR of a full-column-rank A (a different routine
    than the oracle's SVD)."""
    Q, _ = np.linalg.qr(A)
    return np.sum(Q ** 2, axis=1)


def test_leverage_full_rank_tall():
    A = np.random.default_rng(0).standard_normal((40, 7))
    ell = orc.leverage_scores(A)
    np.testing.assert_allclose(ell, _hat_diag_qr(A), rtol=1e-12, atol=1e-14)
    assert abs(ell.sum() - 7) < 1e-12
    assert np.all(ell >= 0) and np.all(ell <= 1 + 1e-12)
    # invariant under an invertible column transformation (depends on range(A) only)
    T = np.random.default_rng(1).standard_normal((7, 7))
    np.testing.assert_allclose(orc.leverage_scores(A @ T), ell, rtol=1e-9, atol=1e-12)


def test_leverage_rank_deficient_and_wide():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((30, 4))
    A = np.concatenate([B, B[:, :2] * 3.0, B @ rng.standard_normal((4, 3))], axis=1)  # rank 4
    ell = orc.leverage_scores(A)
    assert abs(ell.sum() - 4) < 1e-10
    np.testing.assert_allclose(ell, _hat_diag_qr(B), rtol=1e-9, atol=1e-12)
    W = rng.standard_normal((3, 10))               # wide, full row rank -> all ones
    np.testing.assert_allclose(orc.leverage_scores(W), np.ones(3), rtol=1e-12)
    E = np.zeros((5, 2))
    E[1, 0] = 2.0
    E[3, 1] = -1.0                                 # [e_1, e_3] scaled: leverage on rows 1, 3
    np.testing.assert_allclose(orc.leverage_scores(E), [0, 1, 0, 1, 0], atol=1e-15)
    with pytest.raises(ValueError):
        orc.leverage_scores(np.zeros((4, 3)))


def test_core_distribution():
    core = np.random.default_rng(4).standard_normal((3, 50, 4))
    p, cdf = orc.core_distribution(core)
    assert abs(p.sum() - 1) < 1e-14
    assert np.all(np.diff(cdf) >= 0)
    assert abs(cdf[-1] - 1) < 1e-13
    np.testing.assert_allclose(p * 12, _hat_diag_qr(orc.core_unfold2(core)), rtol=1e-10)


def test_inverse_cdf_rules():
    p = np.array([0.25, 0.25, 0.0, 0.5])
    cdf = np.cumsum(p)
    u = np.array([0.0, 0.2499, 0.25, 0.4999, 0.5, 0.75, 0.999999])
    np.testing.assert_array_equal(orc.inverse_cdf(cdf, p, u), [0, 0, 1, 1, 3, 3, 3])
    # rounding left cdf[-1] < 1 and u above it: the largest index with p > 0
    p2 = np.array([0.5, 0.5 - 1e-12, 0.0])
    cdf2 = np.cumsum(p2)
    assert orc.inverse_cdf(cdf2, p2, np.array([1.0 - 1e-13]))[0] == 1


def _product_q(ps, dims, n):
    N = len(dims)
    others = orc.ring_modes(N, n)
    grids = list(itertools.product(*[range(dims[m]) for m in others]))
    idx = np.array(grids)
    q = np.ones(len(grids))
    for m, mode in enumerate(others):
        q *= ps[mode][idx[:, m]]
    lin = orc.ring_linear_index(idx, dims, n)
    out = np.zeros(int(np.prod([dims[m] for m in others])))
    out[lin] = q
    return out


def test_sampler_frequencies_and_weights():
    dims = (3, 4, 5)
    rng = np.random.default_rng(5)
    ps = [rng.uniform(0.1, 1.0, d) for d in dims]
    ps = [p / p.sum() for p in ps]
    ps[2][1] = 0.0
    ps[2] /= ps[2].sum()
    cdfs = [np.cumsum(p) for p in ps]
    n, J = 0, 200000
    idx, w = orc.draw_samples(ps, cdfs, n, J, seed=9, update_id=3)
    q = _product_q(ps, dims, n)
    lin = orc.ring_linear_index(idx, dims, n)
    counts = np.bincount(lin, minlength=q.size)
    assert counts[q == 0].sum() == 0                       # zero-probability cells never drawn
    pos = q > 0
    assert stats.chisquare(counts[pos], J * q[pos]).pvalue > 1e-4
    np.testing.assert_allclose(w ** 2 * J * q[lin], 1.0, rtol=1e-13)   # Def. 5 rescaling


def test_sketch_is_unbiased():
    """E[S^T S] = I for S ~ D(J, q) (Def. 5): the mean of sum_j w_j^2 [v_j = i] is 1."""
    dims = (2, 3, 4)
    rng = np.random.default_rng(6)
    ps = [rng.uniform(0.2, 1.0, d) for d in dims]
    ps = [p / p.sum() for p in ps]
    cdfs = [np.cumsum(p) for p in ps]
    n, J, T = 1, 40, 3000
    K = dims[0] * dims[2]
    acc = np.zeros(K)
    for t in range(T):
        idx, w = orc.draw_samples(ps, cdfs, n, J, seed=17, update_id=t)
        acc += np.bincount(orc.ring_linear_index(idx, dims, n), weights=w ** 2, minlength=K)
    mean = acc / T
    q = _product_q(ps, dims, n)
    sd = np.sqrt((1.0 / q - 1.0) / J / T)      # std of the mean of a scaled binomial
    assert np.all(np.abs(mean - 1.0) < 5 * sd)


def test_lemma35_leverage_bound():
    """Lemma 6 / its proof: ell_i(G_[2]^{!=n}) <= prod_{j!=n} ell_{i_j}(G_(2)^(j)), hence
    q^{!=n} >= beta_n * p with p the exact leverage distribution of G_[2]^{!=n}."""
    dims, ranks = (5, 4, 6, 3), (2, 3, 2, 2)
    rng = np.random.default_rng(7)
    N = len(dims)
    cores = [rng.standard_normal((ranks[(k - 1) % N], dims[k], ranks[k])) for k in range(N)]
    ps = [orc.core_distribution(c)[0] for c in cores]
    ells = [orc.leverage_scores(orc.core_unfold2(c)) for c in cores]
    for n in range(N):
        G2 = orc.subchain_unfold2(cores, n)
        ell = orc.leverage_scores(G2)
        prod_ell = _product_q(ells, dims, n)
        assert np.all(ell <= prod_ell + 1e-12)
        p_exact = ell / ell.sum()
        beta = 1.0 / (ranks[n - 1] * ranks[n] *
                      np.prod([ranks[j] ** 2 for j in range(N) if j not in (n, (n - 1) % N)]))
        assert np.all(_product_q(ps, dims, n) >= beta * p_exact - 1e-15)


# ----------------------------------------------------------------------------------------
# Uniform sampling (the Sec. 5 alternative to leverage scores).
# ----------------------------------------------------------------------------------------
def _uniform_ps(dims):
    return [np.full(d, 1.0 / d) for d in dims]


def test_uniform_sampler_frequencies_and_weights():
    """Every cell of prod_{j!=n} I_j is drawn with probability 1/prod I_j (chi-square), and
    w^2 J q = 1 with q taken from the brute-force product of the uniform marginals."""
    dims = (3, 4, 5)
    n, J = 1, 200000
    idx, w = orc.draw_samples_uniform(dims, n, J, seed=9, update_id=3)
    for m, mode in enumerate(orc.ring_modes(3, n)):
        assert idx[:, m].min() >= 0 and idx[:, m].max() < dims[mode]
    q = _product_q(_uniform_ps(dims), dims, n)
    lin = orc.ring_linear_index(idx, dims, n)
    counts = np.bincount(lin, minlength=q.size)
    assert stats.chisquare(counts, J * q).pvalue > 1e-4
    np.testing.assert_allclose(w ** 2 * J * q[lin], 1.0, rtol=1e-13)


def test_uniform_sketch_is_unbiased():
    """E[S^T S] = I under uniform sampling (Def. 5 with q = 1 / prod I_j)."""
    dims = (2, 3, 4)
    n, J, T = 2, 30, 3000
    K = dims[0] * dims[1]
    acc = np.zeros(K)
    for t in range(T):
        idx, w = orc.draw_samples_uniform(dims, n, J, seed=23, update_id=t)
        acc += np.bincount(orc.ring_linear_index(idx, dims, n), weights=w ** 2, minlength=K)
    mean = acc / T
    sd = np.sqrt((K - 1.0) / J / T)
    assert np.all(np.abs(mean - 1.0) < 5 * sd)


def test_uniform_draws_equal_inverse_cdf_of_uniform_distributions():
    """With uniform marginals p = 1/I the leverage sampler (inverse CDF, pinned above) and
    the uniform sampler take the same uniforms to the same indices and weights."""
    dims = (7, 300, 5, 2)
    n, J = 3, 50000
    ps = _uniform_ps(dims)
    cdfs = [np.arange(1, d + 1) / d for d in dims]
    idx_l, w_l = orc.draw_samples(ps, cdfs, n, J, seed=77, update_id=2 ** 33 + 1)
    idx_u, w_u = orc.draw_samples_uniform(dims, n, J, seed=77, update_id=2 ** 33 + 1)
    np.testing.assert_array_equal(idx_u, idx_l)
    np.testing.assert_allclose(w_u, w_l, rtol=1e-15)


def test_uniform_index_clamps_at_the_top():
    """floor(u * I) is I - 1 for the largest representable u < 1 (no index I)."""
    u = np.array([1.0 - 2.0 ** -53])
    for I in (1, 3, 2 ** 31 - 1):
        assert int(np.minimum(np.floor(u * I), I - 1.0)[0]) == I - 1
