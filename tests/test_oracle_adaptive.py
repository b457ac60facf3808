"""Pins for the oracle's adaptive-sample-size pieces (Sec. 4.2): a sample size per core
update, and merging repeated draws into one weighted row. CPU only."""

import numpy as np
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs


def _small_draws(J=400, seed=3):
    dims, ranks = (3, 4, 5), (2, 2, 2)
    cores = [c.numpy() for c in inputs.random_cores(dims, ranks, 11)]
    ps, cdfs = zip(*[orc.core_distribution(c) for c in cores])
    idx, w = orc.draw_samples(list(ps), list(cdfs), 2, J, seed, 7)    # 3 x 4 = 12 cells
    return dims, ranks, cores, idx, w


def test_merge_counts_weights_and_order_by_brute_force():
    _, _, _, idx, w = _small_draws()
    mi, mw, cnt = orc.merge_duplicates(idx, w)
    # brute force: walk the draws, first occurrence defines the order
    seen, order, counts = {}, [], {}
    for j, row in enumerate(map(tuple, idx)):
        if row not in seen:
            seen[row] = j
            order.append(row)
        counts[row] = counts.get(row, 0) + 1
    assert [tuple(r) for r in mi] == order
    assert list(cnt) == [counts[r] for r in order]
    assert int(np.sum(cnt)) == idx.shape[0] and len(order) < idx.shape[0]
    for r, wm in zip(order, mw):
        assert wm == w[seen[r]] * np.sqrt(float(counts[r]))


def test_merge_leaves_the_normal_equations_unchanged():
    """c copies of a row with weight w and one copy with weight sqrt(c) w give the same
    A^T A and A^T Y (the reason merging is allowed)."""
    dims, ranks, cores, idx, w = _small_draws(600, 5)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=2, rel_noise=1e-2, dtype=torch.float64)
    A = orc.sampled_subchain(cores, 2, idx, w)
    Y = orc.sampled_fibres(X.numpy(), 2, idx, w)
    mi, mw, _ = orc.merge_duplicates(idx, w)
    Am = orc.sampled_subchain(cores, 2, mi, mw)
    Ym = orc.sampled_fibres(X.numpy(), 2, mi, mw)
    assert Am.shape[0] < A.shape[0]
    np.testing.assert_allclose(Am.T @ Am, A.T @ A, rtol=1e-12, atol=1e-12 * np.abs(A.T @ A).max())
    np.testing.assert_allclose(Am.T @ Ym, A.T @ Y, rtol=1e-12, atol=1e-12 * np.abs(A.T @ Y).max())


def test_merged_driver_equals_unmerged():
    dims, ranks = (8, 9, 7), (2, 3, 2)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=4, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 5)]
    a = orc.tr_als_sampled(X.numpy(), init, 300, 3, 6, solver="normal")
    b = orc.tr_als_sampled(X.numpy(), init, 300, 3, 6, solver="normal", merge=True)
    for x, y in zip(a, b):
        np.testing.assert_allclose(y, x, rtol=1e-9, atol=1e-12)


def test_per_update_schedule():
    dims, ranks = (10, 9, 8), (2, 3, 2)
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=6, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 7)]
    # constant within each sweep: the per-sweep schedule, bit for bit
    a = orc.tr_als_sampled(X.numpy(), init, [[200] * 3, [300] * 3], 2, 8, solver="normal")
    b = orc.tr_als_sampled(X.numpy(), init, [200, 300], 2, 8, solver="normal")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # an update's sample size changes that update and what follows, never what precedes it
    c = orc.tr_als_sampled(X.numpy(), init, [[200, 250, 300]], 1, 8, solver="normal")
    d = orc.tr_als_sampled(X.numpy(), init, [[200, 250, 301]], 1, 8, solver="normal")
    assert np.array_equal(c[0], d[0]) and np.array_equal(c[1], d[1])
    assert not np.array_equal(c[2], d[2])
    e = orc.tr_als_sampled(X.numpy(), init, [[200, 251, 300]], 1, 8, solver="normal")
    assert np.array_equal(c[0], e[0]) and not np.array_equal(c[1], e[1])
