"""Pins for the oracle's tensor-ring format, unfoldings and subchains (Sec. 3.1, eq. 1,
Def. 2, Def. 3, the objective identity of Sec. 3.1 and Remark 1). CPU only."""

import itertools
import os

import numpy as np
import pytest

import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_cores(dims, ranks, seed):
    rng = np.random.default_rng(seed)
    N = len(dims)
    return [rng.standard_normal((ranks[(k - 1) % N], dims[k], ranks[k])) for k in range(N)]


def _brute_tr(cores):
    """eq. (1) term by term: sum over every r of the product of core entries."""
    N = len(cores)
    dims = [G.shape[1] for G in cores]
    ranks = [G.shape[2] for G in cores]
    X = np.zeros(dims)
    for i in itertools.product(*[range(d) for d in dims]):
        tot = 0.0
        for r in itertools.product(*[range(R) for R in ranks]):
            prod = 1.0
            for n in range(N):
                prod *= cores[n][r[n - 1], i[n], r[n]]     # r_{n-1} with r_{-1} = r_{N-1}
            tot += prod
        X[i] = tot
    return X


@pytest.mark.parametrize("dims,ranks", [((3, 4, 2), (2, 3, 2)), ((2, 3, 2, 3), (2, 1, 3, 2)),
                                        ((4, 3), (2, 3))])
def test_reconstruct_matches_bruteforce(dims, ranks):
    cores = _rand_cores(dims, ranks, 1)
    np.testing.assert_allclose(orc.tr_reconstruct(cores), _brute_tr(cores), rtol=1e-12,
                               atol=1e-12)


def test_remark1_tt_ranks():
    vals = {}
    for line in open(os.path.join(GOLDEN, "remark1_tr_vs_tt.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        vals[k] = [int(x) for x in v]
    a, i, b = np.meshgrid(np.arange(2), np.arange(2), np.arange(2), indexing="ij")
    G = (1 + a + 2 * i + 4 * b).astype(np.float64)          # reshape(1:8,2,2,2), column-major
    X = orc.tr_reconstruct([G, G, G, G])
    tt = []
    for k in range(1, 4):
        tt.append(int(np.linalg.matrix_rank(X.reshape(2 ** k, 2 ** (4 - k)))))
    assert tt == vals["tt_ranks"]
    assert 4 * G.size == vals["tr_params"][0]
    assert 2 * (2 * 2) + 2 * (2 * 2 * 4) == vals["tt_params"][0]


def test_unfoldings_elementwise():
    rng = np.random.default_rng(3)
    dims = (2, 3, 4, 5)
    X = rng.standard_normal(dims)
    N = len(dims)
    for n in range(N):
        Xc = orc.unfold_classical(X, n)
        Xr = orc.unfold_ring(X, n)
        for i in itertools.product(*[range(d) for d in dims]):
            # classical: other modes in natural order, first fastest
            col, stride = 0, 1
            for m in range(N):
                if m != n:
                    col += i[m] * stride
                    stride *= dims[m]
            assert Xc[i[n], col] == X[i]
            # ring: n+1, ..., N-1, 0, ..., n-1, first fastest
            col, stride = 0, 1
            for m in list(range(n + 1, N)) + list(range(n)):
                col += i[m] * stride
                stride *= dims[m]
            assert Xr[i[n], col] == X[i]


def test_subchain_matches_definition():
    dims, ranks = (2, 3, 2, 3), (2, 3, 1, 2)
    cores = _rand_cores(dims, ranks, 5)
    N = len(dims)
    for n in range(N):
        T = orc.subchain_full(cores, n)
        others = orc.ring_modes(N, n)
        assert T.shape == (ranks[n], int(np.prod([dims[m] for m in others])), ranks[n - 1])
        for ii in itertools.product(*[range(dims[m]) for m in others]):
            lin = int(orc.ring_linear_index(np.array([ii]), dims, n)[0])
            for rn in range(ranks[n]):
                for rm in range(ranks[n - 1]):
                    # Def. 3: sum over all r except r_{n-1}, r_n of prod_{j != n} G^(j)
                    tot = 0.0
                    free = [j for j in range(N) if j not in (n, (n - 1) % N)]
                    for rf in itertools.product(*[range(ranks[j]) for j in free]):
                        r = [None] * N
                        r[n], r[(n - 1) % N] = rn, rm
                        for j, v in zip(free, rf):
                            r[j] = v
                        prod = 1.0
                        for j in range(N):
                            if j == n:
                                continue
                            idx_j = ii[others.index(j)]
                            prod *= cores[j][r[j - 1], idx_j, r[j]]
                        tot += prod
                    assert abs(T[rn, lin, rm] - tot) < 1e-12


@pytest.mark.parametrize("dims,ranks", [((4, 5, 3), (2, 3, 2)), ((3, 2, 4, 3), (2, 2, 3, 1))])
def test_objective_identity(dims, ranks):
    """||TR - X||_F = ||G_[2]^{!=n} G_(2)^(n)T - X_[n]^T||_F (Sec. 3.1), and more strongly the
    unfolded reconstruction equals the product elementwise."""
    cores = _rand_cores(dims, ranks, 7)
    X = np.random.default_rng(8).standard_normal(dims)
    T = orc.tr_reconstruct(cores)
    lhs = np.linalg.norm(T - X)
    for n in range(len(dims)):
        G2 = orc.subchain_unfold2(cores, n)
        Gn = orc.core_unfold2(cores[n])
        np.testing.assert_allclose(G2 @ Gn.T, orc.unfold_ring(T, n).T, rtol=1e-12, atol=1e-12)
        rhs = np.linalg.norm(G2 @ Gn.T - orc.unfold_ring(X, n).T)
        assert abs(lhs - rhs) < 1e-10 * lhs


def test_core_unfold_roundtrip():
    core = np.random.default_rng(0).standard_normal((3, 5, 4))
    Z = orc.core_unfold2(core).T
    np.testing.assert_array_equal(orc.core_from_solution(Z, 3, 4), core)
    # column overline{r_{n-1} r_n} = r_{n-1} + R_{n-1} r_n
    G2 = orc.core_unfold2(core)
    assert G2[2, 1 + 3 * 2] == core[1, 2, 2]


def test_sampled_rows_are_rows_of_full_subchain():
    dims, ranks = (3, 4, 2, 3), (2, 3, 2, 2)
    cores = _rand_cores(dims, ranks, 11)
    X = np.random.default_rng(12).standard_normal(dims)
    rng = np.random.default_rng(13)
    N = len(dims)
    for n in range(N):
        others = orc.ring_modes(N, n)
        J = 17
        idx = np.stack([rng.integers(0, dims[m], J) for m in others], axis=1)
        w = rng.uniform(0.5, 2.0, J)
        lin = orc.ring_linear_index(idx, dims, n)
        full = orc.subchain_unfold2(cores, n)
        np.testing.assert_allclose(orc.sampled_subchain(cores, n, idx, w),
                                   full[lin] * w[:, None], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(orc.sampled_fibres(X, n, idx, w),
                                   orc.unfold_ring(X, n).T[lin] * w[:, None], rtol=0, atol=0)
