"""The benchmark's headline workload end to end against the oracle: 500 x 500 x 500 FP32
X = TR(rank-10 N(0,1) cores) + noise of norm 1e-2 ||TR||, target ranks 10, J = 4000, 10 sweeps,
mixed precision, the benchmark's seeds. The final relative error (Sec. 5.1) must be within 1%
of the oracle's (FP64, the paper's QR-based LS step) from the same start and sample seed."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_headline_final_error_matches_the_oracle():
    wl = inputs.WORKLOADS["tr3_500_r10_fp32"]
    dims, ranks, J, sweeps = wl["dims"], wl["ranks"], wl["J"], wl["sweeps"]
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=wl["seed"], rel_noise=wl["rel_noise"],
                                dtype=torch.float32)
    init = inputs.random_cores(dims, ranks, wl["init_seed"])
    Xn = X.numpy().astype(np.float64)
    ref = orc.tr_als_sampled(Xn, [c.numpy() for c in init], J, sweeps, wl["sample_seed"])
    e_o = orc.rel_error(ref, Xn)
    del Xn
    ctx = T.Context(0)
    try:
        Xd = X.to(DEV)
        out = T.empty_cores(dims, ranks, device=DEV)
        T.tr_als_sampled(ctx, Xd, ranks, J, sweeps, wl["sample_seed"], T.TR_PREC_MIXED, out,
                         init_cores=[inputs.slice_major(c).to(DEV) for c in init])
        e_g = T.tr_rel_error(ctx, Xd, ranks, out)
    finally:
        ctx.close()
    assert abs(e_g - e_o) <= 0.01 * e_o, (e_g, e_o)
