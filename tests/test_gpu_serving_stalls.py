"""Served requests that end near relative error 1 are stalls of the method, not of the
serving layer: for three 4- and 5-way request shapes of the serving workload (ranks 6..12,
J = 10 max L, random N(0,1) starts, stop rule of Sec. 4.1 with tolerance 1e-4, cap 20 sweeps),
the oracle's stopped driver (FP64, no singular step) ends at relative errors above 1 too, and
the FP64 server follows it: same sweep count, final error within 1%, no singular update."""

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

SHAPES = [((19, 22, 21, 17), (9, 11, 11, 9), 1210),
          ((9, 17, 9, 18, 11), (7, 10, 10, 12, 10), 1200),
          ((10, 14, 16, 13, 9), (6, 11, 9, 11, 7), 990)]


@pytest.mark.parametrize("dims,ranks,J", SHAPES)
def test_stalled_request_follows_the_oracle(dims, ranks, J):
    X, _ = inputs.tr_plus_noise(dims, ranks, seed=5, rel_noise=1e-2, dtype=torch.float64)
    init = [c.numpy() for c in inputs.random_cores(dims, ranks, 6)]
    _, fits, _ = orc.tr_als_sampled_until(X.numpy(), init, J, 9, 1e-4, 20, solver="normal")
    e_o = 1.0 - fits[-1]
    assert e_o > 0.5, "this shape no longer stalls in the oracle"
    srv = T.Server(max_slots=8, max_modes=5, max_dim=32, max_rank=12, max_samples=J,
                   max_sweeps=20, fit_tol=1e-4, X_dtype=T.TR_F64, prec=T.TR_PREC_FP64,
                   hbm_budget_bytes=1 << 30, arena_bytes=256 << 20)
    try:
        cores = [torch.from_numpy(np.ascontiguousarray(c.transpose(1, 0, 2))).to(DEV)
                 for c in init]
        t = srv.submit(X.to(DEV), ranks, J, 9, cores, init_given=True)
        r = srv.wait(t, timeout_ms=600000)
    finally:
        srv.close()
    assert r["sweeps"] == len(fits)
    assert r["singular_updates"] == 0
    e_s = 1.0 - r["fit"]
    assert abs(e_s - e_o) <= 0.01 * e_o, (e_s, e_o)
