"""The plain FP64 GPU form of TR-ALS-Sampled, used only as the benchmark's comparator.

It runs Alg. 2 with one stock PyTorch FP64 operation per stage and no fusion, no graph
capture and no custom kernels: leverage scores from ``torch.linalg.qr`` of G_(2)^(n),
``torch.multinomial`` draws per mode (Alg. 3), batched slice products (Alg. 4), fibre
indexing, and ``torch.linalg.lstsq`` for the sampled LS. The library path never calls it.
"""

from __future__ import annotations

from typing import List

import torch


def _leverage_p(core: torch.Tensor) -> torch.Tensor:
    Rl, I, Rr = core.shape
    G2 = core.permute(1, 2, 0).reshape(I, Rr * Rl)
    if I >= Rr * Rl:
        Q, _ = torch.linalg.qr(G2, mode="reduced")
        ell = (Q * Q).sum(dim=1)
    else:
        U, s, _ = torch.linalg.svd(G2, full_matrices=False)
        r = int((s > max(G2.shape) * torch.finfo(torch.float64).eps * s[0]).sum())
        ell = (U[:, :r] ** 2).sum(dim=1)
    return ell / ell.sum()


def als_sampled(X: torch.Tensor, init_cores: List[torch.Tensor], J: int, sweeps: int,
                seed: int) -> List[torch.Tensor]:
    """X: device tensor (any float dtype); init_cores: (Rl, I, Rr) FP64 device tensors."""
    N = X.ndim
    dims = list(X.shape)
    cores = [c.clone() for c in init_cores]
    g = torch.Generator(device=X.device)
    g.manual_seed(int(seed))
    ps = [None] * N
    for k in range(1, N):
        ps[k] = _leverage_p(cores[k])
    for _ in range(sweeps):
        for n in range(N):
            modes = [(n + 1 + m) % N for m in range(N - 1)]
            idx = [torch.multinomial(ps[m], J, replacement=True, generator=g) for m in modes]
            q = torch.ones(J, dtype=torch.float64, device=X.device)
            for m, i in zip(modes, idx):
                q = q * ps[m][i]
            w = 1.0 / torch.sqrt(J * q)
            S = cores[modes[0]][:, idx[0], :].permute(1, 0, 2)
            for m, i in zip(modes[1:], idx[1:]):
                S = torch.bmm(S, cores[m][:, i, :].permute(1, 0, 2))
            A = S.reshape(J, -1) * w[:, None]
            ix = [None] * N
            for m, i in zip(modes, idx):
                ix[m] = i[:, None]
            ix[n] = torch.arange(dims[n], device=X.device)[None, :]
            Y = X[tuple(ix)].to(torch.float64) * w[:, None]
            Z = torch.linalg.lstsq(A, Y).solution            # (L, I_n)
            Rl, _, Rr = cores[n].shape
            cores[n] = Z.reshape(Rr, Rl, dims[n]).permute(1, 2, 0).contiguous()
            ps[n] = _leverage_p(cores[n])
    return cores


def rel_error(X: torch.Tensor, cores: List[torch.Tensor]) -> float:
    """||TR - X|| / ||X|| in FP64 with stock ops (3-way: one matmul per leading block)."""
    N = X.ndim
    T = cores[0]
    for G in cores[1:-1]:
        Ra, M, _ = T.shape
        T = torch.einsum("amb,bic->amic", T, G).reshape(Ra, M * G.shape[1], G.shape[2])
    last = cores[-1]
    Ra, M, Rb = T.shape
    lhs = T.permute(1, 0, 2).reshape(M, Ra * Rb)
    rhs = last.permute(2, 0, 1).reshape(Ra * Rb, last.shape[1])
    Xf = X.reshape(M, -1)
    se, sx = 0.0, 0.0
    step = max(1, (1 << 26) // max(1, rhs.shape[1]))
    for s in range(0, M, step):
        blk = Xf[s:s + step].to(torch.float64)
        d = blk - lhs[s:s + step] @ rhs
        se += float((d * d).sum())
        sx += float((blk * blk).sum())
    return (se / sx) ** 0.5
