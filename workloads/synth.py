"""Seeded synthetic inputs shaped like the workloads of arXiv 1607.07395.

This module only draws inputs. It holds none of the method's arithmetic (no
sampling of indices, no sketching, no clustering), so both the GPU library's
tests and the FP64 oracle may use it.

The paper's datasets (Table 1, Section 5: two sparse rating/text matrices and
two dense images) are not available here, so these generators stand in for
them with the shapes and value distributions of the five benchmark
configurations:

* ``plain_lowrank``     A = U V^T + E, U (m x r), V (n x r) i.i.d. N(0,1),
                        E i.i.d. N(0, noise_var); stored FP64 row-major.
* ``rbf_mixture``       points x_i, y_j in R^d from a Gaussian mixture; the
                        matrix entries exp(-|x_i - y_j|^2 / 2 sigma^2) are
                        never stored; sigma = median distance over 1000 pairs.
* ``decaying_lowrank``  A = U diag(s) V^T + N(0, noise_std^2), U and V
                        orthonormalised Gaussian, s_i = exp(-i / decay).
* ``sparse_lowrank``    compressed-row sparse matrices like Table 1's sparse data
                        (power-law row and column popularity, rank-r values).
* ``batched_specs``     per-member (m, n, rank, k) for the batched workload.

Random draws use numpy's Philox bit generator keyed by (seed, 3) on the host,
or a seeded ``torch.Generator`` on the GPU for the multi-GiB matrices.
"""
from __future__ import annotations

import numpy as np

DATA_TAG = 3  # Philox key word 1 reserved for input generation


def host_rng(seed: int, stream: int = 0) -> np.random.Generator:
    """numpy Generator over Philox4x64-10 keyed by (seed, DATA_TAG)."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, DATA_TAG], dtype=np.uint64)
    ctr = np.array([0, stream, 0, 0], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key, counter=ctr))


def plain_lowrank(m: int = 2000, n: int = 1500, r: int = 20, noise_var: float = 1e-6,
                  seed: int = 1607) -> np.ndarray:
    """A = U V^T + E in FP64 (the plain FP64 workload: 2000 x 1500, rank 20).

    The noise variance 1e-6 is read as a variance (std 1e-3)."""
    g = host_rng(seed)
    U = g.standard_normal((m, r))
    V = g.standard_normal((n, r))
    E = g.standard_normal((m, n)) * np.sqrt(noise_var)
    return np.ascontiguousarray(U @ V.T + E)


def exact_lowrank_int(m: int, n: int, r: int, seed: int = 7, lo: int = -3, hi: int = 3) -> np.ndarray:
    """An exactly rank-r FP64 matrix L R^T with small-integer factors (exact in FP64)."""
    g = host_rng(seed, stream=1)
    L = g.integers(lo, hi + 1, size=(m, r)).astype(np.float64)
    R = g.integers(lo, hi + 1, size=(n, r)).astype(np.float64)
    return np.ascontiguousarray(L @ R.T)


def rbf_mixture(m: int = 100000, n: int = 100000, d: int = 16, components: int = 50,
                seed: int = 1607, sigma_pairs: int = 1000):
    """Points for the implicit RBF kernel matrix.

    Mixture: ``components`` means drawn N(0, 4 I) (std 2), unit-variance
    isotropic components, equal weights (the weights are not stated; equal is
    the reading). x and y are drawn independently from the same mixture.
    sigma is the median of |x_a - y_b| over ``sigma_pairs`` uniformly drawn
    (a, b) pairs. Returns (X float32 m x d, Y float32 n x d, sigma float32).
    """
    g = host_rng(seed, stream=2)
    means = 2.0 * g.standard_normal((components, d))
    cx = g.integers(0, components, size=m)
    cy = g.integers(0, components, size=n)
    X = (means[cx] + g.standard_normal((m, d))).astype(np.float32)
    Y = (means[cy] + g.standard_normal((n, d))).astype(np.float32)
    a = g.integers(0, m, size=sigma_pairs)
    b = g.integers(0, n, size=sigma_pairs)
    dist = np.sqrt(((X[a].astype(np.float64) - Y[b].astype(np.float64)) ** 2).sum(axis=1))
    sigma = np.float32(np.median(dist))
    return np.ascontiguousarray(X), np.ascontiguousarray(Y), sigma


def decaying_lowrank_host(m: int, n: int, rank: int = 256, decay: float = 30.0,
                          noise_std: float = 1e-4, seed: int = 1607, dtype=np.float32):
    """Host version of A = U diag(s) V^T + noise for sizes that fit in host memory.

    Returns (A, U, s, V) with A in ``dtype`` row-major and the FP64 factors of
    the noiseless part L = U diag(s) V^T."""
    g = host_rng(seed, stream=3)
    rank = min(rank, m, n)
    U, _ = np.linalg.qr(g.standard_normal((m, rank)))
    V, _ = np.linalg.qr(g.standard_normal((n, rank)))
    s = np.exp(-np.arange(1, rank + 1) / decay)
    A = (U * s) @ V.T + noise_std * g.standard_normal((m, n))
    return np.ascontiguousarray(A.astype(dtype)), U, s, V


def decaying_lowrank_device(m: int, n: int, rank: int = 256, decay: float = 30.0,
                            noise_std: float = 1e-4, seed: int = 1607, device="cuda",
                            out=None, row_block: int = 8192, noise_fp32: bool = False):
    """Device version of A = U diag(s) V^T + noise in FP32 (e.g. 65536 x 32768, 8 GiB).

    U and V are Gaussian matrices (drawn on the device) orthonormalised by a
    LAPACK QR in FP64 on the host (torch's device linear algebra is not needed,
    so the generator also runs under a profiler); the product is formed in
    FP64 one row block at a time and rounded to FP32. ``out`` may be a
    preallocated (m x lda) FP32 device tensor whose first n columns are
    filled. noise_fp32 draws the noise in FP32 (faster, for the many matrices
    of the batched and serving workloads). Returns (A, U, s, V) with the FP64
    factors on the device."""
    import torch

    def orthonormal(rows):
        g = torch.randn(rows, rank, generator=gen, device=device, dtype=torch.float64)
        q, _ = np.linalg.qr(g.cpu().numpy())
        return torch.from_numpy(np.ascontiguousarray(q)).to(device)

    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + 17)
    rank = min(rank, m, n)
    U = orthonormal(m)
    V = orthonormal(n)
    s = torch.exp(-torch.arange(1, rank + 1, device=device, dtype=torch.float64) / decay)
    A = out if out is not None else torch.empty(m, n, device=device, dtype=torch.float32)
    Us = U * s
    for r0 in range(0, m, row_block):
        r1 = min(m, r0 + row_block)
        blk = Us[r0:r1] @ V.T
        ndt = torch.float32 if noise_fp32 else torch.float64
        blk += noise_std * torch.randn(r1 - r0, n, generator=gen, device=device, dtype=ndt)
        A[r0:r1, :n].copy_(blk)
        del blk
    return A, U, s, V


def sketch_factors(m: int, n: int, k: int, rank: int | None = None, seed: int = 11, s_range: float = 1e-3,
                   dup: bool = False):
    """Factors shaped like a sketching output: U (m x k) and V (n x k) with
    Gaussian unit-norm columns, S geometric from 1 down to s_range, columns
    and S entries beyond `rank` zero; with dup, column 1 of U repeats column 0."""
    g = host_rng(seed, 5)
    r = k if rank is None else rank
    U = g.standard_normal((m, k))
    V = g.standard_normal((n, k))
    U /= np.linalg.norm(U, axis=0)
    V /= np.linalg.norm(V, axis=0)
    S = np.geomspace(1.0, s_range, k) if k > 1 else np.ones(1)
    U[:, r:] = 0.0
    V[:, r:] = 0.0
    S[r:] = 0.0
    if dup and r > 1:
        U[:, 1] = U[:, 0]
    return U, S, V


def sparse_lowrank(m: int = 27000, n: int = 46000, density: float = 0.0056, rank: int = 20,
                   seed: int = 1607, kind: str = "ratings", alpha: float = 0.5):
    """A sparse matrix in compressed rows shaped like Table 1's sparse data:
    "ratings" (27000 x 46000, 0.56 %: values on a 0.5-step scale from 0.5 to
    5 around a rank-`rank` model) or "text" (18774 x 61188, 0.22 %: positive
    log-normal weights scaled by a rank-`rank` non-negative model).

    Row and column popularity follow power laws (weights (i + 1)^-alpha in a
    random order), as rating and term counts do; each row draws its columns
    with those weights, duplicates removed. Returns (indptr int64 m + 1,
    indices int32 sorted within rows, data float32)."""
    g = host_rng(seed, 6)
    nnz_target = int(round(density * m * n))
    rw = (np.arange(1, m + 1, dtype=np.float64) ** -alpha)[g.permutation(m)]
    cw = (np.arange(1, n + 1, dtype=np.float64) ** -alpha)[g.permutation(n)]
    deg = np.maximum(1, np.minimum(n // 2, np.round(rw / rw.sum() * nnz_target).astype(np.int64)))
    pc = cw / cw.sum()
    key = np.zeros(0, dtype=np.int64)
    for _ in range(3):  # top rows up to their degree (repeated popular columns collapse)
        have = np.bincount(key // n, minlength=m) if len(key) else np.zeros(m, dtype=np.int64)
        need = np.maximum(deg - have, 0)
        if need.sum() == 0:
            break
        r = np.repeat(np.arange(m, dtype=np.int64), need)
        c = g.choice(n, size=len(r), p=pc).astype(np.int64)
        key = np.sort(np.concatenate([key, r * n + c]))
        key = key[np.r_[True, key[1:] != key[:-1]]]
    rows, cols = key // n, key % n
    U = g.standard_normal((m, rank)) / np.sqrt(rank)
    V = g.standard_normal((n, rank))
    base = np.empty(len(rows))
    for s0 in range(0, len(rows), 1 << 20):
        s1 = min(len(rows), s0 + (1 << 20))
        base[s0:s1] = np.einsum("ij,ij->i", U[rows[s0:s1]], V[cols[s0:s1]])
    if kind == "ratings":
        vals = np.clip(np.round((3.5 + base + 0.5 * g.standard_normal(len(rows))) * 2) / 2, 0.5, 5.0)
    else:
        vals = np.exp(0.5 * g.standard_normal(len(rows))) * np.log1p(np.abs(base) + 1.0)
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr, cols.astype(np.int32), vals.astype(np.float32)


def batched_specs(count: int = 512, seed: int = 1607, lo: int = 1000, hi: int = 20000,
                  rank_lo: int = 10, rank_hi: int = 100, k_lo: int = 16, k_hi: int = 128):
    """Per-member (m, n, rank, k) for the batched workload: m, n ~ U[lo, hi],
    rank ~ U[rank_lo, rank_hi], k ~ U[k_lo, k_hi] (all inclusive integers)."""
    g = host_rng(seed, stream=4)
    m = g.integers(lo, hi + 1, size=count)
    n = g.integers(lo, hi + 1, size=count)
    rank = g.integers(rank_lo, rank_hi + 1, size=count)
    k = g.integers(k_lo, k_hi + 1, size=count)
    return [dict(m=int(a), n=int(b), rank=int(c), k=int(d)) for a, b, c, d in zip(m, n, rank, k)]
