"""The cluster FP64 Cholesky (n <= 144) and the one-CTA Cholesky give identical factors:
the LS solve (mode 0, including a singular normal matrix) and the leverage distribution
(mode 1, tall and wide cores) are bit-identical under both forms. The cluster form is
selected with TRALS_CHOL_CLUSTER=1 in a child process."""

import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2010_08581_gb300 import inputs
from paper_2010_08581_gb300 import trals as T
dev = "cuda:0"
ctx = T.Context(0)
out = {}
g = torch.Generator().manual_seed(5)
for (J, Rl, Rr, I) in [(4000, 10, 10, 500), (300, 4, 4, 70), (2000, 12, 12, 90),
                       (1500, 8, 9, 333)]:
    L = Rl * Rr
    A = torch.randn(J, L, generator=g, dtype=torch.float64).to(dev)
    Y = torch.randn(J, I, generator=g, dtype=torch.float64).to(dev)
    for prec, dt in ((T.TR_PREC_FP64, torch.float64), (T.TR_PREC_MIXED, torch.float32)):
        core = torch.zeros(I, Rl, Rr, dtype=torch.float64, device=dev)
        T.tr_solve(ctx, A.to(dt), Y.to(dt), Rl, Rr, prec, core)
        out[f"solve_{L}_{I}_{prec}"] = core.cpu()
A0 = torch.randn(50, 36, generator=g, dtype=torch.float64)
A0[:, 7] = 0.0                                   # singular normal matrix: core kept
core = torch.full((40, 6, 6), 3.0, dtype=torch.float64, device=dev)
try:
    T.tr_solve(ctx, A0.to(dev), torch.randn(50, 40, generator=g, dtype=torch.float64).to(dev),
               6, 6, T.TR_PREC_FP64, core)
    T.tr_status_sync(ctx)
    out["singular_status"] = torch.tensor([0])
except T.TrError as e:
    out["singular_status"] = torch.tensor([e.status])
out["singular_core"] = core.cpu()
for (I, Rl, Rr) in [(500, 10, 10), (60, 12, 12), (7, 4, 5), (144, 12, 12)]:
    c = torch.randn(I, Rl, Rr, generator=g, dtype=torch.float64).to(dev)
    p = torch.empty(I, dtype=torch.float64, device=dev)
    cdf = torch.empty(I, dtype=torch.float64, device=dev)
    T.tr_leverage(ctx, c, p, cdf)
    T.tr_status_sync(ctx)
    out[f"lev_{I}_{Rl * Rr}"] = torch.stack([p, cdf]).cpu()
torch.save(out, sys.argv[2])
"""


def _run(tmp_path, name, cluster):
    env = dict(os.environ)
    env.pop("TRALS_CHOL_CLUSTER", None)
    if cluster:
        env["TRALS_CHOL_CLUSTER"] = "1"
    path = str(tmp_path / name)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, path], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return torch.load(path)


def test_cluster_and_one_cta_cholesky_agree_bitwise(tmp_path):
    a = _run(tmp_path, "one_cta.pt", False)
    b = _run(tmp_path, "cluster.pt", True)
    assert a.keys() == b.keys()
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert int(a["singular_status"][0]) == 4            # TR_ERR_SINGULAR
    assert torch.all(a["singular_core"] == 3.0)        # the core was kept
