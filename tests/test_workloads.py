"""The seeded synthetic inputs follow their stated recipes (CPU only): the
plain low-rank matrix's rank and noise level, the decaying spectrum and its
orthonormal factors, the RBF mixture's bandwidth rule, the sparse matrices'
density, order and rating scale, and the batched members' ranges."""
import numpy as np

from workloads import synth


def test_plain_lowrank_rank_and_noise():
    A = synth.plain_lowrank(400, 300, r=5, noise_var=1e-6, seed=3)
    assert A.dtype == np.float64 and A.shape == (400, 300) and A.flags["C_CONTIGUOUS"]
    s = np.linalg.svd(A, compute_uv=False)
    # five Gaussian rank-one terms of size ~ sqrt(m n), then noise of std 1e-3:
    # the largest noise singular value is about 1e-3 (sqrt(m) + sqrt(n)) = 0.037
    assert s[4] > 100 and s[5] < 0.05
    assert np.array_equal(A, synth.plain_lowrank(400, 300, r=5, noise_var=1e-6, seed=3))
    assert not np.array_equal(A, synth.plain_lowrank(400, 300, r=5, noise_var=1e-6, seed=4))


def test_decaying_lowrank_spectrum_and_noise():
    A, U, s, V = synth.decaying_lowrank_host(600, 400, rank=50, decay=10, noise_std=1e-4, seed=5)
    assert A.dtype == np.float32 and A.shape == (600, 400)
    assert np.allclose(U.T @ U, np.eye(50), atol=1e-12) and np.allclose(V.T @ V, np.eye(50), atol=1e-12)
    assert np.allclose(s, np.exp(-np.arange(1, 51) / 10.0), rtol=0, atol=0)
    E = A.astype(np.float64) - (U * s) @ V.T
    # the noise (and the FP32 rounding, far below it) has std 1e-4
    assert abs(E.std() / 1e-4 - 1) < 0.02 and abs(E.mean()) < 1e-6


def test_rbf_mixture_bandwidth_rule():
    X, Y, sigma = synth.rbf_mixture(3000, 2000, d=16, components=7, seed=9, sigma_pairs=500)
    assert X.dtype == np.float32 and Y.dtype == np.float32 and X.shape == (3000, 16) and Y.shape == (2000, 16)
    assert isinstance(sigma, np.float32) and sigma > 0
    # sigma is a median of point distances: about half of random pairs lie closer
    g = np.random.default_rng(0)
    a, b = g.integers(0, 3000, 4000), g.integers(0, 2000, 4000)
    d = np.sqrt(((X[a].astype(np.float64) - Y[b]) ** 2).sum(axis=1))
    assert 0.4 < (d < sigma).mean() < 0.6
    X2, Y2, s2 = synth.rbf_mixture(3000, 2000, d=16, components=7, seed=9, sigma_pairs=500)
    assert np.array_equal(X, X2) and np.array_equal(Y, Y2) and sigma == s2


def test_sparse_ratings_shape():
    m, n, dens = 2000, 3000, 0.01
    ip, ix, v = synth.sparse_lowrank(m, n, dens, rank=8, seed=2)
    assert ip.dtype == np.int64 and ix.dtype == np.int32 and v.dtype == np.float32
    assert ip[0] == 0 and ip[-1] == len(ix) == len(v) and np.all(np.diff(ip) >= 1)  # every row has an entry
    nnz = len(v)
    assert abs(nnz / (dens * m * n) - 1) < 0.15
    for r in range(0, m, 97):  # sorted, distinct, in range within each row
        c = ix[ip[r]:ip[r + 1]]
        assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < n
    # ratings on the half-step scale 0.5 .. 5
    assert v.min() >= 0.5 and v.max() <= 5.0 and np.all(v * 2 == np.round(v * 2))
    # power-law popularity: the busiest rows hold far more entries than the median row
    deg = np.diff(ip)
    assert deg.max() > 5 * np.median(deg)


def test_sparse_text_values_positive():
    ip, ix, v = synth.sparse_lowrank(1000, 2000, 0.005, rank=5, seed=4, kind="text")
    assert np.all(v > 0) and ip[-1] == len(v)


def test_batched_specs_ranges():
    specs = synth.batched_specs(count=300, seed=11)
    assert len(specs) == 300
    m = np.array([s["m"] for s in specs])
    r = np.array([s["rank"] for s in specs])
    k = np.array([s["k"] for s in specs])
    assert m.min() >= 1000 and m.max() <= 20000 and r.min() >= 10 and r.max() <= 100
    assert k.min() >= 16 and k.max() <= 128
    assert specs == synth.batched_specs(count=300, seed=11)


def test_decaying_lowrank_device_generator_on_cpu():
    """The generator of the dense benchmark matrix (run here on torch's CPU
    device, in row blocks and into a wider preallocated buffer, as the bench
    uses it): the same recipe as the host version."""
    import torch
    out = torch.zeros(700, 520, dtype=torch.float32)
    A, U, s, V = synth.decaying_lowrank_device(700, 500, rank=40, decay=30, noise_std=1e-4, seed=7, device="cpu",
                                               out=out, row_block=256)
    assert A is out and torch.all(out[:, 500:] == 0)
    U, s, V = U.numpy(), s.numpy(), V.numpy()
    assert np.allclose(U.T @ U, np.eye(40), atol=1e-12) and np.allclose(V.T @ V, np.eye(40), atol=1e-12)
    assert np.allclose(s, np.exp(-np.arange(1, 41) / 30.0), rtol=1e-15, atol=0)
    E = out[:, :500].double().numpy() - (U * s) @ V.T
    assert abs(E.std() / 1e-4 - 1) < 0.02
