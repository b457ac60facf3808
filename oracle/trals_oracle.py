"""FP64 NumPy oracle of TR-ALS-Sampled and TR-ALS (Malik & Becker, "A Sampling-Based
Method for Tensor Ring Decomposition", ICML 2021).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py``; never by the CUDA library or its binding.

Conventions (0-based; the paper is 1-based):
  * ``cores[k]`` has the paper's shape ``(R_{k-1}, I_k, R_k)`` = ``(Rl_k, I_k, Rr_k)``
    (Sec. 3.1, eq. 1), with ``ranks[k]`` the paper's ``R_{k+1}`` and ``R_{-1} = R_{N-1}``.
  * ``X`` is a NumPy array of shape ``dims`` (C order). Where the paper's linear index
    ``overline{i_1 ... i_N}`` appears (Sec. 3 notation, Def. 2, Def. 3) it is taken
    with the FIRST listed index fastest, as the paper defines it.
  * Ring order of the other modes for core ``n``: ``n+1, ..., N-1, 0, ..., n-1``
    (Def. 2, Def. 3, eq. for q).

Every function names the passage it follows. Steps use only NumPy library primitives
(matmul, einsum, cumsum, searchsorted, SVD, QR, Cholesky, triangular solve) in the order
the paper states them.

Parity pins: every function below is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, published known-answer vectors or brute force; none is
"parity unpinned".
"""

from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

__all__ = [
    "philox4x32_10", "philox_uniforms", "ring_modes", "ring_linear_index",
    "tr_reconstruct", "rel_error", "unfold_classical", "unfold_ring",
    "core_unfold2", "core_from_solution", "subchain_full", "subchain_unfold2",
    "leverage_scores", "core_distribution", "inverse_cdf", "draw_samples",
    "draw_samples_uniform", "merge_duplicates",
    "sampled_subchain", "sampled_fibres", "sampled_ls_normal", "sampled_ls_normal_drop",
    "sampled_ls_qr",
    "sampled_core_update", "tr_als_sampled", "tr_als_sampled_until", "tr_als", "tr_als_update",
]

# --------------------------------------------------------------------------------------
# Counter-based random numbers: Philox4x32-10, from its published definition
# (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
# The paper leaves the generator unspecified (Alg. 3 only says "draw"); this one is
# used so that the CUDA sampler and this oracle can draw the same stream.
# --------------------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
    as easy as 1, 2, 3", SC 2011), the counter-based generator behind the draws of Alg. 3;
    the paper leaves the generator open.

    ``ctr``: integer array of shape (..., 4) (32-bit words); ``key``: two 32-bit words.
    One round maps (c0, c1, c2, c3) to (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
    hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the key is bumped by the Weyl constants (W0, W1)
    between rounds.
    """
    ctr = np.asarray(ctr, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = (ctr[..., i] for i in range(4))
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
            k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0), p1 & _MASK32,
                          (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1), p0 & _MASK32)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def philox_uniforms(J, m, seed, update_id):
    """Uniform variates u in [0, 1) for samples j = 0..J-1 at ring position m (the
    independent draws of Alg. 3, one per sample and sampled mode).

    Counter = (j, m // 2, low32(update_id), high32(update_id)); key = (low32(seed),
    high32(seed)). Position m takes the word pair (2*(m % 2), 2*(m % 2) + 1) of the block
    as (hi, lo) and maps the top 53 bits of hi*2^32 + lo to u = bits * 2^-53.
    """
    j = np.arange(J, dtype=np.uint64)
    ctr = np.stack([j,
                    np.full(J, m // 2, np.uint64),
                    np.full(J, update_id & 0xFFFFFFFF, np.uint64),
                    np.full(J, (update_id >> 32) & 0xFFFFFFFF, np.uint64)], axis=-1)
    out = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)).astype(np.uint64)
    q = m % 2
    bits = ((out[:, 2 * q] << np.uint64(32)) | out[:, 2 * q + 1]) >> np.uint64(11)
    return bits.astype(np.float64) * 2.0 ** -53


# --------------------------------------------------------------------------------------
# Tensor ring format and unfoldings
# --------------------------------------------------------------------------------------
def ring_modes(N, n):
    """Modes other than n in ring order n+1, ..., N-1, 0, ..., n-1 (Def. 2)."""
    return [(n + 1 + m) % N for m in range(N - 1)]


def ring_linear_index(multi, dims, n):
    """overline{i_{n+1} ... i_N i_1 ... i_{n-1}} with the first listed index fastest
    (Sec. 3 notation, used by Def. 2/3 and eq. for q). ``multi`` is (J, N-1) in ring
    order."""
    multi = np.asarray(multi, dtype=np.int64)
    lin = np.zeros(multi.shape[0], dtype=np.int64)
    stride = 1
    for m, mode in enumerate(ring_modes(len(dims), n)):
        lin += multi[:, m] * stride
        stride *= dims[mode]
    return lin


def tr_reconstruct(cores):
    """Full tensor of a tensor ring, eq. (1): X(i_1..i_N) = trace(prod_n G^(n)(:, i_n, :)).

    Cores are merged left to right (matmul over the shared rank index); the trace closes
    the ring with the last core."""
    dims = [G.shape[1] for G in cores]
    T = np.asarray(cores[0], dtype=np.float64)          # (R_{N-1}, I_0, R_0)
    for G in cores[1:-1]:
        Ra, M, _ = T.shape
        T = np.einsum("amb,bic->amic", T, G).reshape(Ra, M * G.shape[1], G.shape[2])
    if len(cores) == 1:
        X = np.einsum("aia->i", T)
    else:
        X = np.einsum("amb,bia->mi", T, cores[-1])
    return X.reshape(dims)


def rel_error(cores, X):
    """Relative error ||TR(cores) - X||_F / ||X||_F (Sec. 5.1)."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm(tr_reconstruct(cores) - X) / np.linalg.norm(X))


def unfold_classical(X, n):
    """Classical mode-n unfolding X_(n), Def. 2: column index overline{i_1..i_{n-1}
    i_{n+1}..i_N}, first listed index fastest."""
    N = X.ndim
    order = [n] + [m for m in range(N) if m != n]
    return np.transpose(X, order).reshape(X.shape[n], -1, order="F")


def unfold_ring(X, n):
    """Mode-n unfolding X_[n], Def. 2: column index overline{i_{n+1}..i_N i_1..i_{n-1}},
    first listed index fastest."""
    order = [n] + ring_modes(X.ndim, n)
    return np.transpose(X, order).reshape(X.shape[n], -1, order="F")


def core_unfold2(core):
    """Classical mode-2 unfolding G_(2)^(n) of a core (R_{n-1}, I_n, R_n): row i_n, column
    overline{r_{n-1} r_n} = r_{n-1} + R_{n-1} r_n (Def. 2)."""
    Rl, I, Rr = core.shape
    return np.transpose(core, (1, 2, 0)).reshape(I, Rr * Rl)


def core_from_solution(Z, Rl, Rr):
    """Inverse of ``core_unfold2``: Z is G_(2)^(n)T of shape (R_{n-1} R_n, I_n), the
    solution of the LS step of Alg. 2 written back as core n (Def. 2)."""
    L, I = Z.shape
    assert L == Rl * Rr
    return np.ascontiguousarray(Z.reshape(Rr, Rl, I).transpose(1, 2, 0))


def subchain_full(cores, n):
    """Subchain tensor G^{!=n}, Def. 3: shape (R_n, prod_{j!=n} I_j, R_{n-1}), middle index
    overline{i_{n+1}..i_{n-1}} with the first listed index fastest. Built by merging the
    other cores in ring order; each new mode becomes the slowest part of the index."""
    N = len(cores)
    modes = ring_modes(N, n)
    T = np.asarray(cores[modes[0]], dtype=np.float64)    # (R_n, I_{n+1}, R_{n+1})
    for mode in modes[1:]:
        G = cores[mode]
        Ra, M, _ = T.shape
        T = np.einsum("amb,bic->aimc", T, G).reshape(Ra, G.shape[1] * M, G.shape[2])
    return T


def subchain_unfold2(cores, n):
    """G_[2]^{!=n}: row = middle index of G^{!=n}, column overline{r_{n-1} r_n}
    (Def. 2 applied to Def. 3)."""
    T = subchain_full(cores, n)                        # (R_n, M, R_{n-1})
    Rn, M, Rm = T.shape
    return np.transpose(T, (1, 0, 2)).reshape(M, Rn * Rm)


# --------------------------------------------------------------------------------------
# Leverage scores and sampling distributions (Def. 4, eq. for p^(n), eq. for q^{!=n})
# --------------------------------------------------------------------------------------
def leverage_scores(A):
    """ell_i(A) = ||U(i, :)||_2^2, U = left singular vectors of A for its rank (Def. 4).

    Numerical rank: singular values above max(K, L) * eps * s_max (the paper states no
    tolerance; this is the usual LAPACK-style choice)."""
    A = np.asarray(A, dtype=np.float64)
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        raise ValueError("zero matrix has no leverage scores (the paper assumes cores != 0)")
    tol = max(A.shape) * np.finfo(np.float64).eps * s[0]
    r = int(np.count_nonzero(s > tol))
    return np.sum(U[:, :r] ** 2, axis=1)


def core_distribution(core):
    """p^(n)(i) = ell_i(G_(2)^(n)) / rank(G_(2)^(n)) (eq. for p^(n)); the divisor is taken
    as sum_i ell_i, which equals the rank (Sec. 3.2). Returns (p, cdf) with cdf the
    sequential inclusive prefix sum in index order."""
    ell = leverage_scores(core_unfold2(core))
    p = ell / np.sum(ell)
    cdf = np.cumsum(p)
    return p, cdf


def inverse_cdf(cdf, p, u):
    """Index i ~ p for uniforms u (the per-mode draws of Alg. 3, Def. 5): smallest i
    with u < cdf[i]; if rounding leaves u >= cdf[-1], the largest i with p[i] > 0."""
    i = np.searchsorted(cdf, u, side="right")
    over = i >= len(cdf)
    if np.any(over):
        last = int(np.nonzero(np.asarray(p) > 0)[0][-1])
        i = np.where(over, last, i)
    return i.astype(np.int64)


def draw_samples(ps, cdfs, n, J, seed, update_id):
    """Draw J i.i.d. multi-indices from q^{!=n} (Alg. 3): i_j ~ p^(j) independently for each
    j != n, in ring order. Returns idx (J, N-1) in ring order and the rescaling
    w = 1 / sqrt(J q^{!=n}(i)) of Def. 5 (product taken in ring order)."""
    N = len(ps)
    modes = ring_modes(N, n)
    idx = np.empty((J, N - 1), dtype=np.int64)
    for m, mode in enumerate(modes):
        u = philox_uniforms(J, m, seed, update_id)
        idx[:, m] = inverse_cdf(cdfs[mode], ps[mode], u)
    q = np.ones(J, dtype=np.float64)
    for m, mode in enumerate(modes):
        q = q * ps[mode][idx[:, m]]
    w = 1.0 / np.sqrt(float(J) * q)
    return idx, w


def draw_samples_uniform(dims, n, J, seed, update_id):
    """Draw J i.i.d. multi-indices from the uniform distribution q^{!=n} = 1 / prod_{j!=n} I_j,
    the alternative to leverage-score sampling of Sec. 5 (uniform sampling experiment).
    Each ring position m takes the same Philox uniform u as the leverage sampler and maps it
    to the index floor(u * I) of a uniform draw on {0, ..., I-1} (clamped to I-1 should
    rounding give I). The rescaling of Def. 5 is the same for every sample:
    w = 1 / sqrt(J q) = sqrt(P / J) with P = prod_{j!=n} I_j, formed in ring order.
    Returns idx (J, N-1) in ring order and w (J,)."""
    N = len(dims)
    modes = ring_modes(N, n)
    idx = np.empty((J, N - 1), dtype=np.int64)
    P = 1.0
    for m, mode in enumerate(modes):
        I = float(dims[mode])
        u = philox_uniforms(J, m, seed, update_id)
        idx[:, m] = np.minimum(np.floor(u * I), I - 1.0).astype(np.int64)
        P = P * I
    w = np.full(J, np.sqrt(P / float(J)), dtype=np.float64)
    return idx, w


def merge_duplicates(idx, w):
    """Merge repeated draws (Sec. 4.2): rows of the sketch that come from the same
    multi-index are identical and carry the same rescaling w (Def. 5 depends only on the
    multi-index), so the c copies of a row contribute c * w^2 a a^T to the normal equations,
    which one row with weight sqrt(c) * w contributes as well. Returns (idx, w, counts) with
    one row per distinct multi-index, in the order of first occurrence."""
    idx = np.asarray(idx, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    _, first, inverse, counts = np.unique(idx, axis=0, return_index=True, return_inverse=True,
                                          return_counts=True)
    order = np.argsort(first, kind="stable")
    return idx[first[order]], w[first[order]] * np.sqrt(counts[order].astype(np.float64)), \
        counts[order]


def sampled_subchain(cores, n, idx, w):
    """Sketch S G_[2]^{!=n} (Alg. 4): row j is the vectorised product of the sampled lateral
    slices G^(n+1)(:, i_{n+1}, :) ... G^(n-1)(:, i_{n-1}, :) (an R_n x R_{n-1} matrix),
    scaled by w_j = 1/c. Column order overline{r_{n-1} r_n}."""
    N = len(cores)
    modes = ring_modes(N, n)
    S = np.transpose(cores[modes[0]][:, idx[:, 0], :], (1, 0, 2)).astype(np.float64)
    for m, mode in enumerate(modes[1:], start=1):
        S = S @ np.transpose(cores[mode][:, idx[:, m], :], (1, 0, 2))
    J = idx.shape[0]
    A = S.reshape(J, -1)          # S[j, r_n, r_{n-1}] -> column r_{n-1} + R_{n-1} r_n
    return A * np.asarray(w, dtype=np.float64)[:, None]


def sampled_fibres(X, n, idx, w):
    """Sketch S X_[n]^T (Alg. 2, sampling of X): row j is the mode-n fibre of X at the sampled
    indices, scaled by w_j."""
    N = X.ndim
    ix = [None] * N
    for m, mode in enumerate(ring_modes(N, n)):
        ix[mode] = np.asarray(idx[:, m])[:, None]
    ix[n] = np.arange(X.shape[n])[None, :]
    Y = np.asarray(X[tuple(ix)], dtype=np.float64)
    return Y * np.asarray(w, dtype=np.float64)[:, None]


def sampled_ls_normal(A, Y):
    """argmin_Z ||A Z - Y||_F through the normal equations: Cholesky A^T A = L L^T, then
    two triangular solves for all right-hand sides (Alg. 2, LS step; same formulation as
    the GPU path)."""
    M = A.T @ A
    B = A.T @ Y
    Lf = np.linalg.cholesky(M)
    return solve_triangular(Lf.T, solve_triangular(Lf, B, lower=True), lower=False)


def sampled_ls_normal_drop(A, Y, tol_scale):
    """argmin_Z ||A Z - Y||_F of the LS step of Alg. 2 for a possibly rank-deficient A:
    a basic least-squares solution. The normal matrix M = A^T A is factored column by column (Cholesky); a column
    whose pivot is <= tol_scale * max diag(M) is dropped (its unknowns are set to 0 and it
    updates nothing), the others give L L^T = M restricted to the kept columns, and the
    kept unknowns solve L L^T Z_k = (A^T Y)_k. With every column kept this is
    sampled_ls_normal."""
    M = A.T @ A
    B = A.T @ Y
    n = M.shape[0]
    tol = tol_scale * np.max(np.diag(M))
    Lf = np.zeros_like(M)
    keep = np.zeros(n, dtype=bool)
    for k in range(n):
        d = M[k, k] - np.dot(Lf[k, :k], Lf[k, :k])
        if not d > tol:
            continue
        keep[k] = True
        Lf[k, k] = np.sqrt(d)
        Lf[k + 1:, k] = (M[k + 1:, k] - Lf[k + 1:, :k] @ Lf[k, :k]) / Lf[k, k]
    Z = np.zeros_like(B)
    Lk = Lf[np.ix_(keep, keep)]
    if keep.any():
        Z[keep] = solve_triangular(Lk.T, solve_triangular(Lk, B[keep], lower=True), lower=False)
    return Z, keep


def sampled_ls_qr(A, Y):
    """argmin_Z ||A Z - Y||_F of the LS step of Alg. 2 through a thin Householder QR of A
    (the QR-based solve the paper costs in its complexity analysis, Sec. 4.3)."""
    Q, R = np.linalg.qr(A, mode="reduced")
    return solve_triangular(R, Q.T @ Y, lower=False)


def _solve(A, Y, solver):
    """The LS step of Alg. 2 by the named solver: "qr" (the paper's QR-based solve),
    "normal" (normal equations, Cholesky; stops on a singular design) or "normal_drop"
    (normal equations with dependent columns dropped at pivot <= L * eps * max diag(A^T A),
    the basic solution a rank-revealing QR-based solve gives)."""
    if solver == "qr":
        return sampled_ls_qr(A, Y)
    if solver == "normal":
        return sampled_ls_normal(A, Y)
    if solver == "normal_drop":
        return sampled_ls_normal_drop(A, Y, A.shape[1] * np.finfo(np.float64).eps)[0]
    raise ValueError(f"unknown solver {solver!r}")


def sampled_core_update(X, cores, ps, cdfs, n, J, seed, update_id, solver="qr",
                        sampling="leverage", merge=False):
    """One inner iteration of Alg. 2 for core n: draw S, sketch G and X, solve the sampled LS.
    ``sampling="uniform"`` draws S from the uniform distribution instead (Sec. 5, uniform
    sampling; ``ps``/``cdfs`` are then unused). ``merge`` merges repeated draws into one
    weighted row (``merge_duplicates``, Sec. 4.2). Returns (new core, idx, w)."""
    if sampling == "uniform":
        idx, w = draw_samples_uniform(X.shape, n, J, seed, update_id)
    else:
        idx, w = draw_samples(ps, cdfs, n, J, seed, update_id)
    if merge:
        idx, w, _ = merge_duplicates(idx, w)
    A = sampled_subchain(cores, n, idx, w)
    Y = sampled_fibres(X, n, idx, w)
    Z = _solve(A, Y, solver)
    Rl, _, Rr = cores[n].shape
    return core_from_solution(Z, Rl, Rr), idx, w


def _initial_distributions(cores, sampling="leverage"):
    """The distributions of cores 1..N-1 formed before the first sweep (Alg. 2); none under
    uniform sampling, which needs no distribution (Sec. 5)."""
    N = len(cores)
    ps, cdfs = [None] * N, [None] * N
    if sampling == "uniform":
        return ps, cdfs
    for n in range(1, N):
        ps[n], cdfs[n] = core_distribution(cores[n])
    return ps, cdfs


def _sweep(X, cores, ps, cdfs, Js, seed, s, solver, sampling="leverage", merge=False):
    """One pass of the outer loop of Alg. 2: update every core in order n = 0..N-1 with
    Js[n] samples, each followed by its new distribution (leverage sampling only); sweep s,
    core n uses update_id = s * N + n."""
    N = len(cores)
    for n in range(N):
        cores[n], _, _ = sampled_core_update(X, cores, ps, cdfs, n, Js[n], seed, s * N + n,
                                             solver, sampling, merge)
        if sampling != "uniform":
            ps[n], cdfs[n] = core_distribution(cores[n])


def _sweep_sizes(J, sweeps, N):
    """The sample size of every update, Js[s][n] (Sec. 4.2: the sample size can change at any
    point at no cost): J is one size for all updates, a list with one size per sweep, or a
    list of sweeps lists with one size per core update."""
    if np.ndim(J) == 0:
        return [[int(J)] * N for _ in range(sweeps)]
    rows = list(J)
    if len(rows) != sweeps:
        raise ValueError("a J schedule needs one entry per sweep")
    out = []
    for r in rows:
        if np.ndim(r) == 0:
            out.append([int(r)] * N)
        else:
            if len(r) != N:
                raise ValueError("a per-update J schedule needs one entry per core")
            out.append([int(v) for v in r])
    return out


def tr_als_sampled(X, init_cores, J, sweeps, seed, solver="qr", callback=None,
                   sampling="leverage", merge=False):
    """TR-ALS-Sampled (Alg. 2) with a fixed number of sweeps. ``init_cores`` supplies
    G^(2..N) (paper numbering); core 0 is overwritten by its first update. ``J`` is the
    sample size of every update, or a list with one sample size per sweep (Sec. 4.2).
    A list of per-sweep lists gives one sample size per core update. ``merge`` merges
    repeated draws into one weighted row (Sec. 4.2; the normal equations are unchanged).
    The sample block of (sweep s, core n) uses update_id = s * N + n. ``sampling`` is
    "leverage" (Alg. 2 as stated) or "uniform" (the Sec. 5 variant: uniform draws, no
    distributions). ``solver`` names the LS step (see ``_solve``); with "normal_drop" a
    rank-deficient design gets a basic solution, and the next distribution is, as always,
    the leverage of the new core (Alg. 2, "update n-th distribution")."""
    if sampling not in ("leverage", "uniform"):
        raise ValueError(f"unknown sampling {sampling!r}")
    Js = _sweep_sizes(J, sweeps, len(init_cores))
    X = np.asarray(X, dtype=np.float64)
    cores = [np.array(G, dtype=np.float64, copy=True) for G in init_cores]
    ps, cdfs = _initial_distributions(cores, sampling)
    for s in range(sweeps):
        _sweep(X, cores, ps, cdfs, Js[s], seed, s, solver, sampling, merge)
        if callback is not None:
            callback(s, cores)
    return cores


def tr_als_sampled_until(X, init_cores, J, seed, fit_tol, max_sweeps, solver="qr",
                         sampling="leverage"):
    """TR-ALS-Sampled (Alg. 2) terminated by the change of the relative error, the first
    criterion of Sec. 4.1: after sweep s the fit f_s = 1 - ||TR - X||_F / ||X||_F is
    computed exactly; the loop ends after a sweep s >= 2 with |f_s - f_{s-1}| < fit_tol,
    or after ``max_sweeps`` sweeps. Returns (cores, fits, converged)."""
    X = np.asarray(X, dtype=np.float64)
    cores = [np.array(G, dtype=np.float64, copy=True) for G in init_cores]
    ps, cdfs = _initial_distributions(cores, sampling)
    fits = []
    for s in range(max_sweeps):
        _sweep(X, cores, ps, cdfs, [int(J)] * len(cores), seed, s, solver, sampling)
        fits.append(1.0 - rel_error(cores, X))
        if len(fits) >= 2 and abs(fits[-1] - fits[-2]) < fit_tol:
            return cores, fits, True
    return cores, fits, False


def tr_als_update(X, cores, n):
    """One inner iteration of Alg. 1: G^(n) = argmin_Z ||G_[2]^{!=n} Z_(2)^T - X_[n]^T||_F with
    the dense subchain."""
    G2 = subchain_unfold2(cores, n)
    Xn = unfold_ring(np.asarray(X, dtype=np.float64), n)
    Z, *_ = np.linalg.lstsq(G2, Xn.T, rcond=None)
    Rl, _, Rr = cores[n].shape
    return core_from_solution(Z, Rl, Rr)


def tr_als(X, init_cores, sweeps):
    """TR-ALS (Alg. 1) with a fixed number of sweeps."""
    cores = [np.array(G, dtype=np.float64, copy=True) for G in init_cores]
    for _ in range(sweeps):
        for n in range(len(cores)):
            cores[n] = tr_als_update(X, cores, n)
    return cores
