"""Autotuner of the batched driver's launch shapes (``tr_batched_tiles``).

For a batch it times every candidate (samples per warp of the sampling kernel x output tile
of the normal-equation contraction) on scratch copies of the batch's cores, keeps the
fastest, sets it on the context and records it in a JSON table keyed by the batch's size
bucket, so later batches of the same shape reuse it without timing. No candidate changes
any result (the library sums every entry in the same order under each), so tuning only
moves time.

The table lives at ``$TRALS_TUNE_CACHE`` if set, else ``~/.cache/trals/batched_tiles.json``.
"""

from __future__ import annotations

import json
import math
import os
from typing import Dict, List, Optional

import torch

from . import trals as T

SAMPLES_PER_WARP = (1, 2, 4, 8)
CONTRACT_TILES = (64, 32)
CANDIDATES = [(spw, tile) for tile in CONTRACT_TILES for spw in SAMPLES_PER_WARP]


def default_table_path() -> str:
    env = os.environ.get("TRALS_TUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "trals", "batched_tiles.json")


def _pow2(x: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, int(x))))))


def bucket_key(problems, prec: int) -> str:
    """Size bucket of a batch: precision, X dtype, and the instance count and the largest
    L, I and J, each rounded up to a power of two."""
    count = len(problems)
    lmax = imax = jmax = 1
    xdt = "f32"
    for pr in problems:
        X = pr["X"]
        xdt = "f64" if X.dtype == torch.float64 else "f32"
        r = list(pr["ranks"])
        N = len(r)
        lmax = max(lmax, max(r[(k - 1) % N] * r[k] for k in range(N)))
        imax = max(imax, max(int(d) for d in X.shape))
        jmax = max(jmax, int(pr["J"]))
    p = "fp64" if prec == T.TR_PREC_FP64 else "mixed"
    return f"{p}/{xdt}/n{_pow2(count)}/L{_pow2(lmax)}/I{_pow2(imax)}/J{_pow2(jmax)}"


def load_table(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or default_table_path()
    try:
        with open(path) as f:
            t = json.load(f)
        return t if isinstance(t, dict) else {}
    except (OSError, ValueError):
        return {}


def save_table(table: Dict[str, dict], path: Optional[str] = None) -> str:
    path = path or default_table_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return path


def tune_batched(ctx: T.Context, problems: List[dict], prec: int, sweeps: int = 1,
                 reps: int = 2, table_path: Optional[str] = None, force: bool = False) -> dict:
    """Choose and set the launch shapes for batches shaped like ``problems`` (the dicts of
    ``tr_als_sampled_batched``). Returns {"samples_per_warp", "contract_tile", "cached",
    "ms": {candidate: ms per call}}."""
    key = bucket_key(problems, prec)
    table = load_table(table_path)
    if key in table and not force:
        e = table[key]
        T.tr_set_batched_tiles(ctx, e["samples_per_warp"], e["contract_tile"])
        return dict(e, cached=True, key=key)
    scratch = [dict(pr, cores=[c.clone() for c in pr["cores"]]) for pr in problems]
    stream = torch.cuda.current_stream()
    times = {}
    for spw, tile in CANDIDATES:
        T.tr_set_batched_tiles(ctx, spw, tile)
        T.tr_als_sampled_batched(ctx, scratch, sweeps, prec)   # first call captures the graph
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            T.tr_als_sampled_batched(ctx, scratch, sweeps, prec)
        b.record(stream)
        torch.cuda.synchronize()
        times[f"{spw}x{tile}"] = a.elapsed_time(b) / reps
    best = min(CANDIDATES, key=lambda c: times[f"{c[0]}x{c[1]}"])
    T.tr_set_batched_tiles(ctx, best[0], best[1])
    entry = {"samples_per_warp": best[0], "contract_tile": best[1], "ms": times}
    table[key] = entry
    save_table(table, table_path)
    return dict(entry, cached=False, key=key)
