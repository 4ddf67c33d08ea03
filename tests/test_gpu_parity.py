"""GPU parity: each hot-path step through the C ABI against the FP64 oracle on
the same seeded inputs, then whole sketches (Algorithm 2).

Bars: integer work (indices, labels, picks) bit-exact; FP64 factors within
1e-10 relative; FP64 k-means labels identical except rows whose oracle
margin (second best - best squared distance) is below 1e-12 (|x|^2 + best),
which are counted and must be absent on these inputs.
"""
import numpy as np
import pytest

from oracle import cabs_ref as o
from workloads import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1607_07395_gb300 import cabs
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return cabs.Context(0)


@pytest.fixture(scope="module")
def C():
    from paper_1607_07395_gb300 import cabs
    return cabs


DEV = "cuda"


def to_np(t):
    return t.detach().cpu().numpy()


def dev(a):
    """Row-major contiguous device copy of a numpy array."""
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def align_signs(got, want):
    """Flip each column of got to match want's sign (singular vectors are defined up to sign)."""
    s = np.sign((got * want).sum(axis=0))
    s[s == 0] = 1
    return got * s


def near_tie_rows(km, t, X):
    xn = (X * X).sum(axis=1)
    return np.nonzero(km.margin[t] < 1e-12 * (xn + km.best[t]))[0]


# ----------------------------------------------------------------- a1: draw

@pytest.mark.parametrize("seed,tag,N,k", [(1607, 0, 2000, 20), (1607, 1, 1500, 20), (7, 0, 65536, 256),
                                          (7, 1, 32768, 256), (3, 0, 100000, 200), (5, 1, 37, 37), (9, 0, 1, 1),
                                          (11, 1, 2**31 - 2, 4096), (2, 0, 5000, 1000)])
def test_draw_bit_exact(ctx, C, seed, tag, N, k):
    drawn, srt = C.cabs_draw_indices(ctx, seed, tag, N, k)
    want_d, want_s = o.draw_indices(seed, tag, N, k)
    assert to_np(drawn).tolist() == want_d.tolist()
    assert to_np(srt).tolist() == want_s.tolist()


# --------------------------------------------------------------- a2: gather

@pytest.mark.parametrize("dtype,m,n,lda,kr,kc", [(np.float64, 2000, 1500, 1500, 20, 20),
                                                 (np.float32, 777, 1031, 1100, 33, 257 - 1),
                                                 (np.float32, 4096, 2048, 32768, 256, 256),
                                                 (np.float64, 131, 67, 67, 1, 7)])
def test_gather_dense_bit_exact(ctx, C, dtype, m, n, lda, kr, kc):
    g = np.random.default_rng(m + n)
    full = g.standard_normal((m, lda)).astype(dtype)
    Ad = dev(full)[:, :n]
    A = full[:, :n]
    rows = np.sort(g.choice(m, kr, replace=False)).astype(np.int32)
    cols = np.sort(g.choice(n, kc, replace=False)).astype(np.int32)
    for prec in ("fp64", "fp32"):
        if prec == "fp32" and dtype == np.float64:
            continue
        Cm, Rt, W = C.cabs_gather(ctx, C.dense_source(Ad), m, n, dev(rows),
                                  dev(cols), prec=prec)
        Co, Rto, Wo = o.gather_dense(A, rows, cols)
        assert np.array_equal(to_np(Cm).astype(np.float64), Co)
        assert np.array_equal(to_np(Rt).astype(np.float64), Rto)
        assert np.array_equal(to_np(W), Wo)
        assert np.array_equal(to_np(W), to_np(Cm)[rows].astype(np.float64))
        assert np.array_equal(to_np(W), to_np(Rt)[cols].T.astype(np.float64))


def test_gather_rbf(ctx, C):
    X, Y, sig = synth.rbf_mixture(3000, 2500, d=16, components=50)
    Xd, Yd = dev(X), dev(Y)
    g = np.random.default_rng(1)
    rows = np.sort(g.choice(3000, 200, replace=False)).astype(np.int32)
    cols = np.sort(g.choice(2500, 200, replace=False)).astype(np.int32)
    Co, Rto, Wo = o.gather_rbf(X, Y, sig, rows, cols)
    for prec, tol in (("fp64", 1e-14), ("fp32", 2e-6)):
        Cm, Rt, W = C.cabs_gather(ctx, C.rbf_source(Xd, Yd, sig), 3000, 2500, dev(rows),
                                  dev(cols), prec=prec)
        Cm, Rt, W = to_np(Cm).astype(np.float64), to_np(Rt).astype(np.float64), to_np(W)
        assert np.abs(Cm - Co).max() <= tol and np.abs(Rt - Rto).max() <= tol
        assert np.array_equal(W, Cm[rows]) and np.array_equal(W, Rt[cols].T)


# ------------------------------------------------------------- a3/a4: core

def _core_case(kind, seed=0):
    if kind == "plain":
        A = synth.plain_lowrank()
        k = 20
    elif kind == "rankdef":
        A = synth.exact_lowrank_int(300, 250, 7, seed=seed)
        k = 16
    else:
        A, _, _, _ = synth.decaying_lowrank_host(1024, 512, rank=128, decay=30, noise_std=1e-4, seed=seed,
                                                 dtype=np.float64)
        k = 128
    g = np.random.default_rng(seed + 5)
    rows = np.sort(g.choice(A.shape[0], k, replace=False))
    cols = np.sort(g.choice(A.shape[1], k, replace=False))
    return A, rows, cols


@pytest.mark.parametrize("kind", ["plain", "rankdef", "decay"])
@pytest.mark.parametrize("mode", ["pinv", "stabilized"])
def test_sketching_fp64_matches_oracle(ctx, C, kind, mode):
    A, rows, cols = _core_case(kind)
    m, n = A.shape
    Co, Rto, Wo = o.gather_dense(A, rows, cols)
    ref = o.sketching(Co, Rto, Wo, m, n, mode)
    for embed in (False, True):
        out = C.cabs_sketching(ctx, dev(Co), dev(Rto),
                               dev(Wo), m, n, prec="fp64", core=mode, embed=embed)
        assert int(out["rank"].item()) == ref.rank
        sig = to_np(out["sig"])
        assert np.allclose(sig, ref.sig, rtol=1e-12, atol=1e-13 * ref.sig[0])
        S = to_np(out["S"])
        assert np.allclose(S, ref.S, rtol=1e-10, atol=1e-12 * max(ref.S.max(), 1e-300))
        U, V = to_np(out["out1"]), to_np(out["out2"])
        if embed:
            U, V = U / np.where(S > 0, np.sqrt(S), 1), V / np.where(S > 0, np.sqrt(S), 1)
        r = ref.rank
        assert np.allclose(align_signs(U[:, :r], ref.U[:, :r]), ref.U[:, :r], atol=1e-10)
        assert np.allclose(align_signs(V[:, :r], ref.V[:, :r]), ref.V[:, :r], atol=1e-10)
        assert np.all(U[:, r:] == 0) and np.all(V[:, r:] == 0)
        got = (U * S) @ V.T
        want = (ref.U * ref.S) @ ref.V.T
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_sketching_fp32_close(ctx, C):
    A, rows, cols = _core_case("decay")
    m, n = A.shape
    A32 = A.astype(np.float32)
    Co, Rto, Wo = o.gather_dense(A32, rows, cols)
    ref = o.sketching(Co, Rto, Wo, m, n, "stabilized")
    out = C.cabs_sketching(ctx, dev(Co.astype(np.float32)),
                           dev(Rto.astype(np.float32)), dev(Wo), m, n,
                           prec="fp32", core="stabilized")
    got = (to_np(out["out1"]).astype(np.float64) * to_np(out["S"])) @ to_np(out["out2"]).astype(np.float64).T
    want = (ref.U * ref.S) @ ref.V.T
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


# ---------------------------------------------------------- a5: k-means

def _embedding(kind="plain", seed=1607):
    A = synth.plain_lowrank() if kind == "plain" else synth.decaying_lowrank_host(
        2048, 1024, rank=64, decay=20, noise_std=1e-4, seed=seed, dtype=np.float64)[0]
    k = 20 if kind == "plain" else 64
    Ir_d, Ir = o.draw_indices(seed, 0, A.shape[0], k)
    Ic_d, Ic = o.draw_indices(seed, 1, A.shape[1], k)
    Co, Rto, Wo = o.gather_dense(A, Ir, Ic)
    sk = o.sketching(Co, Rto, Wo, *A.shape, "pinv")
    return o.embed(sk.U, sk.S), Ir_d, k


@pytest.mark.parametrize("kind,p", [("plain", 0.0), ("plain", 1.0), ("decay", 0.0), ("decay", 2.0)])
def test_kmeans_fp64_labels_bit_exact(ctx, C, kind, p):
    P, init, k = _embedding(kind)
    iters = 5
    ref = o.weighted_kmeans(P, init[:k], iters, p)
    out = C.cabs_kmeans(ctx, dev(P), dev(init[:k].astype(np.int32)), k,
                        iters, prec="fp64", upsilon_pow=p)
    labels = to_np(out["labels"])
    for t in range(iters):
        ties = near_tie_rows(ref, t, P)
        assert ties.size == 0
        assert np.array_equal(labels[t], ref.labels[t]), t
    assert np.allclose(to_np(out["centres"]), ref.Z, rtol=1e-11, atol=1e-12)
    assert np.allclose(to_np(out["energy"]), ref.energy, rtol=1e-11)
    assert int(out["T"].item()) == int(np.bincount(ref.labels[-1], minlength=k).max())


def test_kmeans_fp32_close(ctx, C):
    P, init, k = _embedding("decay")
    ref = o.weighted_kmeans(P, init[:k], 5, 0.0)
    out = C.cabs_kmeans(ctx, dev(P.astype(np.float32)),
                        dev(init[:k].astype(np.int32)), k, 5, prec="fp32")
    labels = to_np(out["labels"])
    # the first assignment only sees FP32 rounding of the same points
    assert (labels[0] != ref.labels[0]).mean() < 1e-3
    assert abs(to_np(out["energy"])[-1] / ref.energy[-1] - 1) < 1e-3


def test_kmeans_edge_cases(ctx, C):
    # single centre; empty cluster from duplicate initial points; M not a multiple of any tile
    X = np.random.default_rng(0).standard_normal((97, 5))
    X[3] = X[0]
    for init, k2 in (([0], 1), ([0, 3, 10], 3)):
        ref = o.weighted_kmeans(X, init, 3, 0.0)
        out = C.cabs_kmeans(ctx, dev(X), torch.tensor(init, dtype=torch.int32, device=DEV),
                            k2, 3, prec="fp64")
        assert np.array_equal(to_np(out["labels"]), np.array(ref.labels))
        assert np.allclose(to_np(out["centres"]), ref.Z, atol=1e-13)
    out = C.cabs_kmeans(ctx, dev(X), torch.tensor([0, 1], dtype=torch.int32, device=DEV), 2, 0,
                        prec="fp64")
    assert np.array_equal(to_np(out["centres"]), X[[0, 1]])


# ---------------------------------------------------------------- a6: snap

@pytest.mark.parametrize("kind", ["plain", "decay"])
def test_snap_fp64_bit_exact(ctx, C, kind):
    P, init, k = _embedding(kind)
    ref = o.weighted_kmeans(P, init[:k], 5, 0.0)
    order, srt = C.cabs_snap(ctx, dev(P), dev(ref.Z), prec="fp64")
    want_o, want_s = o.snap(P, ref.Z)
    assert to_np(order).tolist() == want_o.tolist()
    assert to_np(srt).tolist() == want_s.tolist()


def test_snap_fallback_when_candidates_taken(ctx, C):
    g = np.random.default_rng(3)
    X = g.standard_normal((300, 6))
    Z = np.repeat(g.standard_normal((2, 6)), [12, 5], axis=0)  # 12 identical centres exhaust a top-8 list
    for prec in ("fp64", "fp32"):
        Xt = dev(X)
        Zt = dev(Z)
        if prec == "fp32":
            Xt, Zt = Xt.float(), Zt.float()
        order, srt = C.cabs_snap(ctx, Xt, Zt, prec=prec)
        want_o, want_s = o.snap(to_np(Xt).astype(np.float64), to_np(Zt).astype(np.float64))
        assert to_np(order).tolist() == want_o.tolist()
        assert len(set(to_np(order).tolist())) == Z.shape[0]


@pytest.mark.parametrize("M", [131072, 131073, 150000])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_snap_taken_set_both_forms(ctx, C, M, prec):
    """The greedy walk keeps the rows taken so far as a bitmap in shared
    memory up to 131072 rows and as an open-addressing set beyond: both forms
    give the oracle's picks (Section 3.2), with repeated centres so that lists
    run out (full scans) and later centres meet rows taken before them."""
    g = np.random.default_rng(M)
    X = g.standard_normal((M, 8))
    base = X[g.choice(M, 6, replace=False)]
    Z = np.concatenate([np.repeat(base[:2], [11, 9], axis=0), base[2:] + 0.01 * g.standard_normal((4, 8)),
                        g.standard_normal((10, 8))])
    dt = np.float64 if prec == "fp64" else np.float32
    Xd, Zd = dev(X.astype(dt)), dev(Z.astype(dt))
    order, srt = C.cabs_snap(ctx, Xd, Zd, prec=prec)
    want_o, want_s = o.snap(X.astype(dt).astype(np.float64), Z.astype(dt).astype(np.float64),
                            tie_rtol=o.SNAP_TIE_RTOL if prec == "fp64" else 2.0 ** -16)
    assert to_np(order).tolist() == want_o.tolist()
    assert to_np(srt).tolist() == want_s.tolist()
    assert len(set(to_np(order).tolist())) == Z.shape[0]


# ------------------------------------------------------- whole sketch (a1-a8)

def _run(ctx, C, src_np, src_dev, m, n, k, iters, seed, prec, mode):
    p = C.make_params(m, n, k, iters=iters, seed=seed, prec=prec, core=mode, flags=C.FLAG_FOLLOW_ERR)
    sk = C.cabs_sketch(ctx, src_dev, p)
    torch.cuda.synchronize()
    return p, sk


@pytest.mark.parametrize("mode", ["pinv", "stabilized"])
def test_plain_fp64_sketch_matches_oracle(ctx, C, mode):
    A = synth.plain_lowrank()
    m, n = A.shape
    Ad = dev(A)
    p, sk = _run(ctx, C, A, C.dense_source(Ad), m, n, 20, 5, 1607, "fp64", mode)
    ref = o.cabs(o.DenseSource(A), 20, iters=5, seed=1607, mode=mode)
    assert to_np(sk.pilot_rows).tolist() == ref.pilot_rows.tolist()
    assert to_np(sk.pilot_cols).tolist() == ref.pilot_cols.tolist()
    assert to_np(sk.rows).tolist() == ref.rows.tolist()
    assert to_np(sk.cols).tolist() == ref.cols.tolist()
    U, S, V = to_np(sk.U), to_np(sk.S), to_np(sk.V)
    want = (ref.final.U * ref.final.S) @ ref.final.V.T
    assert np.linalg.norm((U * S) @ V.T - want) <= 1e-10 * np.linalg.norm(want)
    d = sk.diag()
    assert d.rank_pilot == ref.pilot.rank and d.rank_final == ref.final.rank and d.status == 0
    assert np.allclose(list(d.e_rows)[:5], ref.km_rows.energy, rtol=1e-10)
    assert np.allclose(list(d.e_cols)[:5], ref.km_cols.energy, rtol=1e-10)
    assert abs(d.e_follow_rows - ref.e_follow[0]) <= 1e-10 * ref.e_follow[0]
    err = C.cabs_error(ctx, C.dense_source(Ad), p, sk)
    assert abs(err - o.rel_fro_error_dense(A, ref.final.U, ref.final.S, ref.final.V)) <= 1e-9 * err


def test_rbf_fp64_sketch_matches_oracle(ctx, C):
    X, Y, sig = synth.rbf_mixture(6000, 5000, d=16, components=50)
    Xd, Yd = dev(X), dev(Y)
    src = C.rbf_source(Xd, Yd, sig)
    p, sk = _run(ctx, C, None, src, 6000, 5000, 40, 10, 5, "fp64", "pinv")
    ref = o.cabs(o.RBFSource(X, Y, sig), 40, iters=10, seed=5, mode="pinv")
    assert to_np(sk.pilot_rows).tolist() == ref.pilot_rows.tolist()
    assert to_np(sk.rows).tolist() == ref.rows.tolist()
    assert to_np(sk.cols).tolist() == ref.cols.tolist()
    e_gpu = C.cabs_error(ctx, src, p, sk, samples=200000, seed=3)
    e_ref = o.rel_fro_error_sampled(o.RBFSource(X, Y, sig), ref.final.U, ref.final.S, ref.final.V, 3, 200000)
    assert abs(e_gpu - e_ref) <= 1e-8 * max(e_ref, 1e-30)


def test_fp32_sketch_error_close_to_fp64(ctx, C):
    A, _, _, _ = synth.decaying_lowrank_host(4096, 2048, rank=256, decay=30, noise_std=1e-4, seed=1607)
    m, n = A.shape
    Ad = dev(A)
    ref = o.cabs(o.DenseSource(A), 64, iters=5, seed=1607, mode="stabilized")
    e_ref = o.rel_fro_error_dense(A, ref.final.U, ref.final.S, ref.final.V)
    p, sk = _run(ctx, C, A, C.dense_source(Ad), m, n, 64, 5, 1607, "fp32", "stabilized")
    assert to_np(sk.pilot_rows).tolist() == ref.pilot_rows.tolist()
    e = C.cabs_error(ctx, C.dense_source(Ad), p, sk)
    assert e / e_ref - 1 <= 1e-3, (e, e_ref)


# ------------------------------------------------- a3: the FP64 core SVD alone

def _svd_case(k, kind):
    g = np.random.default_rng(1000 + k)
    if kind == "rand":
        return g.standard_normal((k, k))
    if kind == "graded":
        Uq, _ = np.linalg.qr(g.standard_normal((k, k)))
        Vq, _ = np.linalg.qr(g.standard_normal((k, k)))
        return (Uq * 10.0 ** (-8.0 * np.arange(k) / max(k - 1, 1))) @ Vq.T
    r = max(1, k // 3)
    return g.integers(-3, 4, (k, r)).astype(float) @ g.integers(-3, 4, (k, r)).astype(float).T


@pytest.mark.parametrize("k,kind", [(1, "rand"), (2, "rand"), (20, "rand"), (64, "rand"), (65, "rand"),
                                    (128, "graded"), (200, "rand"), (256, "graded"), (256, "rankdef"),
                                    (97, "rankdef")])
def test_core_svd_fp64(ctx, C, k, kind):
    W = _svd_case(k, kind)
    out = C.cabs_sketching(ctx, dev(W), dev(W.T), dev(W), k, k, prec="fp64", core="pinv")
    sig, Uw, Vw = to_np(out["sig"]), to_np(out["Uw"]), to_np(out["Vw"])
    r = int(out["rank"].item())
    ref = np.linalg.svd(W, compute_uv=False)
    assert r == int(np.count_nonzero(ref > k * 2.220446049250313e-16 * ref[0]))
    assert np.abs(sig - ref).max() <= 1e-12 * ref[0]
    assert np.abs(Uw[:, :r].T @ Uw[:, :r] - np.eye(r)).max() <= 1e-12
    assert np.abs(Vw[:, :r].T @ Vw[:, :r] - np.eye(r)).max() <= 1e-12
    rec = (Uw[:, :r] * sig[:r]) @ Vw[:, :r].T
    assert np.linalg.norm(rec - W) <= 1e-12 * np.linalg.norm(W)


# ------------------------------------- hard-threshold follow-up (Section 5 (f))

@pytest.mark.parametrize("M,d,k2", [(1, 1, 1), (5000, 20, 20), (70000, 256, 256), (3001, 7, 3001), (1025, 33, 17)])
def test_threshold_fp64_bit_exact(ctx, C, M, d, k2):
    g = np.random.default_rng(M + d)
    X = g.standard_normal((M, d)) * g.uniform(0.5, 2.0, size=(M, 1))
    if M > 20:
        X[10] = X[3]   # equal norms: the lower row wins wherever the cut falls
        X[17] = -X[3]
    got = to_np(C.cabs_threshold(ctx, dev(X), k2, prec="fp64"))
    assert got.tolist() == o.hard_threshold(X, k2).tolist()


def test_threshold_fp32_and_all_equal(ctx, C):
    g = np.random.default_rng(4)
    X = (g.standard_normal((3000, 24)) * g.uniform(0.5, 2.0, size=(3000, 1))).astype(np.float32)
    got = to_np(C.cabs_threshold(ctx, dev(X), 50, prec="fp32"))
    assert got.tolist() == o.hard_threshold(X.astype(np.float64), 50).tolist()
    ones = np.ones((777, 5))
    assert to_np(C.cabs_threshold(ctx, dev(ones), 9, prec="fp64")).tolist() == list(range(9))


@pytest.mark.parametrize("mode", ["pinv", "stabilized"])
def test_plain_fp64_threshold_sketch_matches_oracle(ctx, C, mode):
    A = synth.plain_lowrank()
    m, n = A.shape
    Ad = dev(A)
    p = C.make_params(m, n, 20, iters=5, seed=1607, prec="fp64", core=mode, flags=C.FLAG_HARD_THRESHOLD)
    sk = C.cabs_sketch(ctx, C.dense_source(Ad), p)
    ref = o.cabs(o.DenseSource(A), 20, iters=5, seed=1607, mode=mode, follow="threshold")
    assert to_np(sk.rows).tolist() == ref.rows.tolist()
    assert to_np(sk.cols).tolist() == ref.cols.tolist()
    U, S, V = to_np(sk.U), to_np(sk.S), to_np(sk.V)
    want = (ref.final.U * ref.final.S) @ ref.final.V.T
    assert np.linalg.norm((U * S) @ V.T - want) <= 1e-10 * np.linalg.norm(want)
    d = sk.diag()
    assert d.rank_final == ref.final.rank and d.status == 0 and list(d.e_rows)[:5] == [0.0] * 5
