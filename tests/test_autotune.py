"""Host logic of the batched-driver autotuner: size buckets and the persisted table
(CPU only)."""

import torch

from paper_2010_08581_gb300 import autotune
from paper_2010_08581_gb300 import trals as T


def _prob(dims, ranks, J, dtype=torch.float32):
    return {"X": torch.zeros(dims, dtype=dtype), "ranks": ranks, "J": J}


def test_bucket_rounds_sizes_up_to_powers_of_two():
    probs = [_prob((30, 25, 20), (3, 4, 2), 160), _prob((90, 6, 33), (4, 3, 5), 200)]
    key = autotune.bucket_key(probs, T.TR_PREC_MIXED)
    # count 2, largest L = 20, I = 90, J = 200
    assert key == "mixed/f32/n2/L32/I128/J256"
    key64 = autotune.bucket_key([_prob((10, 10), (2, 2), 8, torch.float64)], T.TR_PREC_FP64)
    assert key64 == "fp64/f64/n1/L4/I16/J8"


def test_table_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tiles.json")
    assert autotune.load_table(path) == {}
    table = {"mixed/f32/n512/L64/I256/J1024": {"samples_per_warp": 2, "contract_tile": 32}}
    autotune.save_table(table, path)
    assert autotune.load_table(path) == table


def test_candidates_cover_the_abi_range():
    assert set(s for s, _ in autotune.CANDIDATES) == {1, 2, 4, 8}
    assert set(t for _, t in autotune.CANDIDATES) == {64, 32}
