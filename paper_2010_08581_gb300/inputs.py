"""Seeded synthetic inputs for TR-ALS-Sampled, shared by the tests, the oracle checks and
the benchmark.

This module draws random numbers and lays them out. To build a tensor from random cores it
contracts the ring once (eq. 1, in ``_ring_tensor``); neither the oracle nor the CUDA path
computes a tested result with that contraction, and it holds no other step of the method
(no leverage scores, draws, design rows, fibres or least-squares solves). Random cores are returned in the paper's shape ``(R_{k-1}, I_k, R_k)``
(Sec. 3.1); ``slice_major`` converts them to the library's ``[I_k][Rl][Rr]`` layout.

Workload recipes (the paper's datasets are not available; these synthetic tensors stand
in for its synthetic experiment of Sec. 5.1.1 and its image-stack workloads):
  * ``tr_plus_noise``: X = TR(cores) + Gaussian noise, cores i.i.d. N(0, 1), noise
    standard deviation ``rel * ||TR||_F / sqrt(prod I)`` so that the total noise norm is
    ``rel * ||TR||_F``.
  * ``cosine_sum``: X = sum over 20 terms of products over modes of
    cos(2 pi f i_k / I_k + phi), f ~ U[0, 4), phi ~ U[0, 2 pi), plus uniform noise
    U[-a, a] with a = 5 % of max |X|.
"""

from __future__ import annotations

import math
from typing import List, Sequence

import torch


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def random_cores(dims: Sequence[int], ranks: Sequence[int], seed: int,
                 dtype=torch.float64) -> List[torch.Tensor]:
    """N(0, 1) cores; core k has shape (ranks[k-1], dims[k], ranks[k])."""
    g = _gen(seed)
    N = len(dims)
    out = []
    for k in range(N):
        shape = (int(ranks[(k - 1) % N]), int(dims[k]), int(ranks[k]))
        out.append(torch.randn(shape, generator=g, dtype=torch.float64).to(dtype))
    return out


def slice_major(core: torch.Tensor) -> torch.Tensor:
    """(Rl, I, Rr) -> contiguous (I, Rl, Rr): each lateral slice G(:, i, :) contiguous."""
    return core.permute(1, 0, 2).contiguous()


def paper_layout(core_slice_major: torch.Tensor) -> torch.Tensor:
    """(I, Rl, Rr) -> (Rl, I, Rr)."""
    return core_slice_major.permute(1, 0, 2).contiguous()


def _ring_tensor(cores: Sequence[torch.Tensor], device, dtype) -> torch.Tensor:
    """Dense tensor of a ring of cores, merged left to right and closed by a trace."""
    dims = [int(c.shape[1]) for c in cores]
    T = cores[0].to(device=device, dtype=dtype)
    for G in cores[1:-1]:
        G = G.to(device=device, dtype=dtype)
        Ra, M, Rb = T.shape
        T = torch.einsum("amb,bic->amic", T, G).reshape(Ra, M * G.shape[1], G.shape[2])
    last = cores[-1].to(device=device, dtype=dtype)
    Ra, M, Rb = T.shape
    # X[m, i] = sum_{a,b} T[a, m, b] * last[b, i, a]  -> one matmul
    lhs = T.permute(1, 0, 2).reshape(M, Ra * Rb)                    # [m, a*Rb + b]
    rhs = last.permute(2, 0, 1).reshape(Ra * Rb, last.shape[1])     # [a*Rb + b, i]
    return (lhs @ rhs).reshape(dims)


def tr_plus_noise(dims, ranks, seed: int, rel_noise: float, device="cpu",
                  dtype=torch.float32):
    """X = TR(cores) + noise of total norm rel_noise * ||TR||_F. Returns (X, cores)."""
    cores = random_cores(dims, ranks, seed)
    X = _ring_tensor(cores, device, torch.float64 if dtype == torch.float64 else torch.float32)
    if rel_noise > 0:
        sigma = rel_noise * float(torch.linalg.vector_norm(X, dtype=torch.float64)) \
            / math.sqrt(X.numel())
        g = torch.Generator(device=X.device)
        g.manual_seed(int(seed) + 7919)
        X.add_(torch.randn(X.shape, generator=g, device=X.device, dtype=X.dtype), alpha=sigma)
    return X.to(dtype), cores


def cosine_sum(dims, seed: int, terms: int = 20, noise_amp: float = 0.05, device="cpu",
               dtype=torch.float32) -> torch.Tensor:
    """Sum of ``terms`` separable products of low-frequency cosines plus uniform noise."""
    g = _gen(seed)
    factors = []
    for I in dims:
        f = torch.rand(terms, generator=g, dtype=torch.float64) * 4.0
        phi = torch.rand(terms, generator=g, dtype=torch.float64) * (2 * math.pi)
        i = torch.arange(I, dtype=torch.float64)[:, None]
        factors.append(torch.cos(2 * math.pi * f[None, :] * i / I + phi[None, :]))
    # Khatri-Rao of the leading half of the modes times that of the trailing half.
    h = len(dims) // 2

    def khatri_rao(mats):
        out = mats[0]
        for Mx in mats[1:]:
            out = (out[:, None, :] * Mx[None, :, :]).reshape(-1, terms)
        return out

    left = khatri_rao(factors[:h]).to(device=device, dtype=torch.float32)
    right = khatri_rao(factors[h:]).to(device=device, dtype=torch.float32)
    X = (left @ right.T).reshape([int(d) for d in dims])
    a = noise_amp * float(X.abs().max())
    gd = torch.Generator(device=X.device)
    gd.manual_seed(int(seed) + 104729)
    X.add_(torch.rand(X.shape, generator=gd, device=X.device, dtype=X.dtype).mul_(2 * a).sub_(a))
    return X.to(dtype)


def coherent_tr(I: int, true_rank: int, seed: int, N: int = 3, spike: float = 20.0,
                noise_sd: float = 0.1, device="cpu", dtype=torch.float32):
    """The randomly generated tensors of the paper's synthetic experiments (Sec. 5): N cores
    of size R' x I x R' with i.i.d. N(0, 1) entries, one entry of each core (chosen uniformly
    at random) set to ``spike`` to raise the coherence of the least-squares problems, combined
    into the full tensor, plus i.i.d. N(0, noise_sd^2) noise. Returns (X, cores)."""
    dims, ranks = [I] * N, [true_rank] * N
    cores = random_cores(dims, ranks, seed)
    g = _gen(seed + 104729)
    for c in cores:
        pos = int(torch.randint(c.numel(), (1,), generator=g))
        c.view(-1)[pos] = spike
    X = _ring_tensor(cores, device, torch.float64 if dtype == torch.float64 else torch.float32)
    if noise_sd > 0:
        gn = torch.Generator(device=X.device)
        gn.manual_seed(int(seed) + 15485863)
        X.add_(torch.randn(X.shape, generator=gn, device=X.device, dtype=X.dtype), alpha=noise_sd)
    return X.to(dtype), cores


# The paper's highly oscillatory functions (Sec. 5), sampled on a uniform grid of I^N points
# of the interval given here (the paper does not state the intervals; see the readings).
OSCILLATORY = {
    "linear_growth": (lambda x: (x + 1.0) * torch.sin(100.0 * (x + 1.0) ** 2), 0.0, 1.0),
    "airy": (lambda x: x ** -0.25 * torch.sin(2.0 * x ** 1.5 / 3.0), 1.0, 100.0),
    "chirp": (lambda x: torch.sin(4.0 / x) * torch.cos(x ** 2), 0.0, 1.0),
}


def oscillatory(name: str, N: int = 10, I: int = 4, dtype=torch.float32) -> torch.Tensor:
    """f(x_k), k = 0 .. I^N - 1, on the uniform grid x_k = a + (b - a)(k + 1) / I^N of
    (a, b], reshaped to an N-way I x ... x I tensor (row-major: the last mode fastest)."""
    f, a, b = OSCILLATORY[name]
    K = I ** N
    x = a + (b - a) * (torch.arange(K, dtype=torch.float64) + 1.0) / K
    return f(x).reshape([I] * N).to(dtype).contiguous()


def random_distribution(I: int, seed: int, zero_frac: float = 0.0) -> torch.Tensor:
    """A probability vector on [I] (FP64); a fraction of entries set exactly to zero."""
    g = _gen(seed)
    p = torch.rand(I, generator=g, dtype=torch.float64) + 0.05
    if zero_frac > 0:
        z = torch.rand(I, generator=g, dtype=torch.float64) < zero_frac
        z[0] = False
        p[z] = 0.0
    return p / p.sum()


# Workloads: (dims, ranks, J, sweeps, relative noise, X dtype).
WORKLOADS = {
    # 3-way 100^3 FP64 TR of rank 5 + 1e-3 noise, J = 2000, 10 sweeps (FP64 path).
    "tr3_100_r5_fp64": dict(dims=(100, 100, 100), ranks=(5, 5, 5), J=2000, sweeps=10,
                           rel_noise=1e-3, dtype=torch.float64, seed=0, init_seed=0,
                           sample_seed=0),
    # 3-way 500^3 FP32 TR of rank 10 + 1e-2 noise, J = 4000, 10 sweeps (mixed path).
    "tr3_500_r10_fp32": dict(dims=(500, 500, 500), ranks=(10, 10, 10), J=4000, sweeps=10,
                            rel_noise=1e-2, dtype=torch.float32, seed=1, init_seed=1,
                            sample_seed=2),
}


def batched_workload(count: int, seed: int, device="cpu", imin=32, imax=200, rmin=3, rmax=8,
                     rel_noise=1e-3, j_factor=10):
    """Independent 3-way FP32 problems: each I_n ~ U{imin..imax}, each rank ~ U{rmin..rmax},
    X = TR(N(0,1) cores) + noise of total norm rel_noise * ||TR||, J = j_factor * max_k L_k.
    Returns a list of dicts (dims, ranks, J, X, seed)."""
    g = _gen(seed)
    out = []
    for i in range(count):
        dims = tuple(int(v) for v in torch.randint(imin, imax + 1, (3,), generator=g))
        ranks = tuple(int(v) for v in torch.randint(rmin, rmax + 1, (3,), generator=g))
        L = max(ranks[(k - 1) % 3] * ranks[k] for k in range(3))
        X, _ = tr_plus_noise(dims, ranks, seed=seed * 100003 + i, rel_noise=rel_noise,
                             device=device, dtype=torch.float32)
        out.append(dict(dims=dims, ranks=ranks, J=j_factor * L, X=X, seed=seed * 7919 + i))
    return out


def serving_requests(count: int, seed: int, modes=(3, 4, 5), emin=1e5, emax=1e8, rmin=4,
                     rmax=16, j_factor=10):
    """Shapes of a stream of decomposition requests: N ~ U(modes); entry count E
    log-uniform in [emin, emax]; I_k = max(2, round(E^(1/N) * exp(g_k - mean(g)))) with
    g_k ~ U[-0.5, 0.5] (so prod I_k stays near E); each rank ~ U{rmin..rmax};
    J = j_factor * max_k L_k. Returns a list of dicts (dims, ranks, J)."""
    g = _gen(seed)
    out = []
    for _ in range(count):
        N = int(modes[int(torch.randint(len(modes), (1,), generator=g))])
        u = float(torch.rand(1, generator=g, dtype=torch.float64))
        E = math.exp(math.log(emin) + u * (math.log(emax) - math.log(emin)))
        gk = torch.rand(N, generator=g, dtype=torch.float64) - 0.5
        gk = gk - gk.mean()
        dims = tuple(max(2, int(round(E ** (1.0 / N) * math.exp(float(v))))) for v in gk)
        ranks = tuple(int(v) for v in torch.randint(rmin, rmax + 1, (N,), generator=g))
        L = max(ranks[(k - 1) % N] * ranks[k] for k in range(N))
        out.append(dict(dims=dims, ranks=ranks, J=j_factor * L))
    return out


def poisson_arrivals(count: int, rate: float, seed: int) -> List[float]:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    g = _gen(seed)
    gaps = -torch.log1p(-torch.rand(count, generator=g, dtype=torch.float64)) / rate
    return torch.cumsum(gaps, 0).tolist()
