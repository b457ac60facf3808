"""The batched driver (many independent problems, one launch per stage): each instance
matches the single-problem driver and the oracle, and its result is the same alone and
in any mix of other instances."""

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


def to_paper(core_dev):
    return np.ascontiguousarray(np.transpose(core_dev.cpu().numpy(), (1, 0, 2)))


def make_problem(dims, ranks, seed, J, xdt, init=True):
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=seed, rel_noise=1e-2, dtype=xdt)
    init_cores = [c.numpy() for c in inputs.random_cores(dims, ranks, seed + 1000)]
    cores = [torch.from_numpy(np.ascontiguousarray(c.transpose(1, 0, 2))).to(DEV)
             for c in init_cores]
    return {"X": X.to(DEV), "Xh": X, "ranks": ranks, "J": J, "seed": seed + 7, "cores": cores,
            "init": init, "init_np": init_cores}


SHAPES = [((30, 25, 20), (3, 4, 2), 200), ((12, 9, 10, 11), (2, 3, 2, 3), 150),
          ((40, 6, 33), (4, 3, 5), 250),          # mode 1: I = 6 < L = 12 (wide)
          ((21, 17), (3, 5), 100)]


def test_batched_fp64_matches_oracle(ctx):
    probs = [make_problem(d, r, 11 + i, J, torch.float64) for i, (d, r, J) in enumerate(SHAPES)]
    sweeps = 2
    T.tr_als_sampled_batched(ctx, probs, sweeps, T.TR_PREC_FP64)
    for pr in probs:
        ref = orc.tr_als_sampled(pr["Xh"].numpy(), pr["init_np"], pr["J"], sweeps, pr["seed"],
                                 solver="normal")
        for k in range(len(ref)):
            assert rel(to_paper(pr["cores"][k]), ref[k]) < 1e-8


def test_batched_matches_single_problem_driver(ctx):
    sweeps = 3
    probs = [make_problem(d, r, 31 + i, J, torch.float32) for i, (d, r, J) in enumerate(SHAPES)]
    singles = []
    for pr in probs:
        out = [c.clone() for c in pr["cores"]]
        T.tr_als_sampled(ctx, pr["X"], pr["ranks"], pr["J"], sweeps, pr["seed"], T.TR_PREC_MIXED,
                         out, init_cores=[c.clone() for c in pr["cores"]])
        singles.append(out)
    T.tr_als_sampled_batched(ctx, probs, sweeps, T.TR_PREC_MIXED)
    for pr, out in zip(probs, singles):
        e_b = T.tr_rel_error(ctx, pr["X"], pr["ranks"], pr["cores"])
        e_s = T.tr_rel_error(ctx, pr["X"], pr["ranks"], out)
        assert abs(e_b - e_s) < 0.01 * e_s


def test_batched_result_is_the_same_alone_and_in_a_mix(ctx):
    sweeps = 2
    alone = make_problem((30, 25, 20), (3, 4, 2), 51, 200, torch.float32)
    T.tr_als_sampled_batched(ctx, [alone], sweeps, T.TR_PREC_MIXED)
    mixed = make_problem((30, 25, 20), (3, 4, 2), 51, 200, torch.float32)
    others = [make_problem(d, r, 61 + i, J, torch.float32) for i, (d, r, J) in enumerate(SHAPES)]
    T.tr_als_sampled_batched(ctx, others[:2] + [mixed] + others[2:], sweeps, T.TR_PREC_MIXED)
    for a, b in zip(alone["cores"], mixed["cores"]):
        assert torch.equal(a, b)


def test_batched_draws_the_same_initial_cores_as_the_single_driver(ctx):
    """Without given initial cores both drivers draw cores 1..N-1 i.i.d. N(0,1) from the
    instance's seed (Philox4x32-10 + Box-Muller, stream = core index): same start, same
    result."""
    pr = make_problem((30, 25, 20), (3, 4, 2), 71, 200, torch.float32, init=False)
    single = [torch.empty_like(c) for c in pr["cores"]]
    T.tr_als_sampled(ctx, pr["X"], pr["ranks"], pr["J"], 2, pr["seed"], T.TR_PREC_MIXED, single)
    T.tr_als_sampled_batched(ctx, [pr], 2, T.TR_PREC_MIXED)
    e_b = T.tr_rel_error(ctx, pr["X"], pr["ranks"], pr["cores"])
    e_s = T.tr_rel_error(ctx, pr["X"], pr["ranks"], single)
    assert np.isfinite(e_b) and abs(e_b - e_s) < 0.01 * e_s
