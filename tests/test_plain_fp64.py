"""The plain FP64 GPU form (paper_2010_08581_gb300/plain_fp64.py), the comparator of the
benchmark's metric, against the oracle: its leverage distribution and relative error equal
the oracle's (Def. 4, eq. for p^(n); Sec. 5.1), and its whole decomposition (Alg. 2, its own
torch.multinomial draws) ends within 2% of the oracle's final error. The starts are the true
cores plus a perturbation, so that both runs converge to the noise floor instead of to
different stalls (ALS from random starts on tiny tensors often stalls)."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs, plain_fp64

DIMS, RANKS = (40, 30, 20), (3, 4, 2)


def _case(seed):
    X, true = inputs.tr_plus_noise(DIMS, RANKS, seed=seed, rel_noise=1e-2, dtype=torch.float64)
    pert = inputs.random_cores(DIMS, RANKS, seed + 10)
    return X, [t + 0.3 * p for t, p in zip(true, pert)]


def test_components_equal_the_oracle():
    X, init = _case(1)
    for c in init:
        p_o, _ = orc.core_distribution(c.numpy())
        np.testing.assert_allclose(plain_fp64._leverage_p(c).numpy(), p_o, rtol=1e-12, atol=0)
    wide = inputs.random_cores((3, 40, 5), (4, 4, 4), 3)[0]      # I = 40 > L = 16: tall
    np.testing.assert_allclose(plain_fp64._leverage_p(wide).numpy(),
                               orc.core_distribution(wide.numpy())[0], rtol=1e-12)
    narrow = inputs.random_cores((5, 6, 7), (4, 4, 4), 4)[1]      # I = 6 < L = 16: wide
    np.testing.assert_allclose(plain_fp64._leverage_p(narrow).numpy(),
                               orc.core_distribution(narrow.numpy())[0], rtol=1e-12)
    e = plain_fp64.rel_error(X, init)
    assert abs(e - orc.rel_error([c.numpy() for c in init], X.numpy())) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_final_error_matches_the_oracle(seed):
    X, init = _case(seed)
    ref = orc.tr_als_sampled(X.numpy(), [c.numpy() for c in init], 400, 6, 5)
    e_o = orc.rel_error(ref, X.numpy())
    Xd = X.to("cuda:0")
    res = plain_fp64.als_sampled(Xd, [c.to("cuda:0") for c in init], 400, 6, 5)
    e_p = plain_fp64.rel_error(Xd, res)
    assert abs(e_p - e_o) <= 0.02 * e_o, (e_p, e_o)
