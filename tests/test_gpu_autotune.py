"""The batched driver's launch shapes: every candidate gives bit-identical cores, invalid
shapes are refused, and the autotuner sets and records its choice."""

import numpy as np
import pytest
import torch

from paper_2010_08581_gb300 import autotune
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SHAPES = [((30, 25, 20), (3, 4, 2), 160), ((40, 6, 33), (4, 3, 5), 200),
          ((12, 9, 10, 11), (2, 3, 2, 3), 150), ((64, 48, 20), (6, 5, 6), 360)]


def _batch(seed):
    probs = []
    for i, (d, r, J) in enumerate(SHAPES):
        X, _ = inputs.tr_plus_noise(d, r, seed=seed + i, rel_noise=1e-2)
        init = [torch.from_numpy(np.ascontiguousarray(c.numpy().transpose(1, 0, 2))).to(DEV)
                for c in inputs.random_cores(d, r, seed + 100 + i)]
        probs.append(dict(X=X.to(DEV), ranks=r, J=J, seed=seed + 7 + i, cores=init, init=True))
    return probs


def test_every_launch_shape_gives_the_same_cores():
    ctx = T.Context(0)
    base = _batch(300)
    ref = None
    for spw, tile in autotune.CANDIDATES:
        T.tr_set_batched_tiles(ctx, spw, tile)
        assert T.tr_get_batched_tiles(ctx) == (spw, tile)
        for prec in (T.TR_PREC_MIXED,):
            probs = [dict(p, cores=[c.clone() for c in p["cores"]]) for p in base]
            T.tr_als_sampled_batched(ctx, probs, 2, prec)
            got = [c.clone() for p in probs for c in p["cores"]]
            if ref is None:
                ref = got
            else:
                assert all(torch.equal(a, b) for a, b in zip(ref, got)), (spw, tile)
    for bad in (0, 9):
        with pytest.raises(T.TrError) as e:
            T.tr_set_batched_tiles(ctx, bad, 64)
        assert e.value.status == T.TR_ERR_INVALID_ARG
    with pytest.raises(T.TrError):
        T.tr_set_batched_tiles(ctx, 4, 48)
    ctx.close()


def test_autotuner_sets_and_records_its_choice(tmp_path):
    ctx = T.Context(0)
    probs = _batch(400)
    path = str(tmp_path / "tiles.json")
    r = autotune.tune_batched(ctx, probs, T.TR_PREC_MIXED, table_path=path)
    assert not r["cached"] and len(r["ms"]) == len(autotune.CANDIDATES)
    assert T.tr_get_batched_tiles(ctx) == (r["samples_per_warp"], r["contract_tile"])
    best = min(r["ms"].values())
    assert r["ms"][f"{r['samples_per_warp']}x{r['contract_tile']}"] == best
    T.tr_set_batched_tiles(ctx, 4, 64)
    again = autotune.tune_batched(ctx, probs, T.TR_PREC_MIXED, table_path=path)
    assert again["cached"]
    assert T.tr_get_batched_tiles(ctx) == (r["samples_per_warp"], r["contract_tile"])
    ctx.close()
