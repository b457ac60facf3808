"""The paper-shaped synthetic inputs (Sec. 5): the coherent random tensor ring (one entry
per core set to 20, N(0, 0.1^2) noise) and the oscillatory functions on 4^10 points."""

import math

import numpy as np
import torch

from paper_2010_08581_gb300 import inputs


def test_coherent_tr_has_one_spike_per_core_and_the_stated_noise():
    X, cores = inputs.coherent_tr(12, 3, seed=5, noise_sd=0.1, dtype=torch.float64)
    assert X.shape == (12, 12, 12)
    for c in cores:
        assert c.shape == (3, 12, 3)
        assert int((c == 20.0).sum()) == 1
    clean, _ = inputs.coherent_tr(12, 3, seed=5, noise_sd=0.0, dtype=torch.float64)
    noise = (X - clean).numpy().ravel()
    assert abs(noise.std() - 0.1) < 0.01 and abs(noise.mean()) < 0.01
    # the clean tensor is the trace of the slice products, entry by entry
    i, j, k = 3, 7, 11
    ref = torch.trace(cores[0][:, i, :] @ cores[1][:, j, :] @ cores[2][:, k, :])
    assert abs(float(clean[i, j, k]) - float(ref)) < 1e-9 * max(1.0, abs(float(ref)))


def test_oscillatory_values_on_the_grid():
    K = 4 ** 10
    for name, (f, a, b) in inputs.OSCILLATORY.items():
        X = inputs.oscillatory(name, dtype=torch.float64)
        assert X.shape == (4,) * 10
        flat = X.reshape(-1)
        for k in (0, 12345, K - 1):
            x = a + (b - a) * (k + 1) / K
            if name == "linear_growth":
                ref = (x + 1) * math.sin(100 * (x + 1) ** 2)
            elif name == "airy":
                ref = x ** -0.25 * math.sin(2 * x ** 1.5 / 3)
            else:
                ref = math.sin(4 / x) * math.cos(x * x)
            assert abs(float(flat[k]) - ref) < 1e-9
