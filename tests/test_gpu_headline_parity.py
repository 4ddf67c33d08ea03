"""GPU FP64 parity at the widths the benchmarks run (k > 64: the cluster SVD
with QR preconditioning, the cluster-sized refinement, k-means and snap at
k up to 256), whole sketches (Algorithm 2) and their steps through the C ABI
against the FP64 oracle on the same seeded inputs.

Bars (FP64 mode): pilot indices, the labels of every k-means iteration and
the follow-up indices bit-exact; k-means rows whose oracle margin is below
1e-12 (|x|^2 + best) would be exempt and are counted (none occur); factors
U diag(S) V^T within 1e-10 relative; the relative error within 1e-9.

The snap's structural ties (the centre of a two-row cluster is equidistant
from both rows: Section 3.2, last paragraph) are decided by the tie window of
the reading, checked here on rows built so that rounding splits the tie
either way.
"""
import numpy as np
import pytest

from oracle import cabs_ref as o
from workloads import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U_FP32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    from paper_1607_07395_gb300 import cabs
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return cabs.Context(0)


@pytest.fixture(scope="module")
def C():
    from paper_1607_07395_gb300 import cabs
    return cabs


def to_np(t):
    return t.detach().cpu().numpy()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def near_ties(km, t, X):
    xn = (X * X).sum(axis=1)
    return int(np.count_nonzero(km.margin[t] < 1e-12 * (xn + km.best[t])))


def check_sketch(C, ctx, src_dev, ref, p, m, n, err_ref, err_samples=0):
    sk = C.cabs_sketch(ctx, src_dev, p)
    torch.cuda.synchronize()
    assert to_np(sk.pilot_rows).tolist() == ref.pilot_rows.tolist()
    assert to_np(sk.pilot_cols).tolist() == ref.pilot_cols.tolist()
    assert to_np(sk.rows).tolist() == ref.rows.tolist()
    assert to_np(sk.cols).tolist() == ref.cols.tolist()
    d = sk.diag()
    assert d.status == 0 and d.rank_pilot == ref.pilot.rank and d.rank_final == ref.final.rank
    it = p.iters
    assert np.allclose(list(d.e_rows)[:it], ref.km_rows.energy, rtol=1e-10)
    assert np.allclose(list(d.e_cols)[:it], ref.km_cols.energy, rtol=1e-10)
    U, S, V = to_np(sk.U), to_np(sk.S), to_np(sk.V)
    got = (U * S) @ V.T
    want = (ref.final.U * ref.final.S) @ ref.final.V.T
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    err = float(to_np(sk.err)[0])
    assert abs(err - err_ref) <= 1e-9 * err_ref, (err, err_ref)
    return sk


def check_steps(C, ctx, ref, P_ref, Q_ref, k, iters):
    """k-means labels of every iteration and the snap, GPU steps on the
    oracle's embeddings."""
    for X, km, drawn, rows_o, rows in ((P_ref, ref.km_rows, ref.pilot_rows_drawn, ref.rows_centre_order, ref.rows),
                                       (Q_ref, ref.km_cols, ref.pilot_cols_drawn, ref.cols_centre_order, ref.cols)):
        out = C.cabs_kmeans(ctx, dev(X), dev(drawn[:k].astype(np.int32)), k, iters, prec="fp64")
        labels = to_np(out["labels"])
        for t in range(iters):
            assert near_ties(km, t, X) == 0
            assert np.array_equal(labels[t], km.labels[t]), t
        order, srt = C.cabs_snap(ctx, dev(X), dev(km.Z), prec="fp64")
        assert to_np(order).tolist() == rows_o.tolist()
        assert to_np(srt).tolist() == rows.tolist()


@pytest.fixture(scope="module")
def dense_slice():
    A = synth.decaying_lowrank_host(4096, 2048, rank=256, seed=1607)[0]
    return A, dev(A)


@pytest.mark.parametrize("k,core,trunc", [(256, "stabilized", 256 * U_FP32), (200, "stabilized", 0.0),
                                          (128, "pinv", 128 * U_FP32), (65, "pinv", 65 * U_FP32)])
def test_dense_fp64_sketch_wide_k_matches_oracle(ctx, C, dense_slice, k, core, trunc):
    """The dense benchmark recipe on its 4096 x 2048 slice (seed 1607, c = 5):
    FP32 A = U diag(exp(-i/30)) V^T + N(0, 1e-4^2), rank 256."""
    A, Ad = dense_slice
    m, n = A.shape
    ref = o.cabs(o.DenseSource(A), k, iters=5, seed=1607, mode=core, trunc_rtol=trunc)
    err_ref = o.rel_fro_error_dense(A, ref.final.U, ref.final.S, ref.final.V)
    p = C.make_params(m, n, k, iters=5, seed=1607, prec="fp64", core=core, trunc_rtol=trunc,
                      flags=C.FLAG_FOLLOW_ERR, err_samples=0)
    check_sketch(C, ctx, C.dense_source(Ad), ref, p, m, n, err_ref)
    check_steps(C, ctx, ref, ref.P, ref.Q, k, 5)


def test_rbf_fp64_sketch_k200_matches_oracle(ctx, C):
    """The implicit RBF recipe (50-component mixture, d = 16) at 6000 x 5000
    points, k = 200, c = 10, the pseudo-inverse core with truncation k 2^-24."""
    X, Y, sig = synth.rbf_mixture(6000, 5000, d=16, components=50)
    k, trunc = 200, 200 * U_FP32
    src = o.RBFSource(X, Y, sig)
    ref = o.cabs(src, k, iters=10, seed=11, mode="pinv", trunc_rtol=trunc)
    err_ref = o.rel_fro_error_sampled(src, ref.final.U, ref.final.S, ref.final.V, 3, 200000)
    p = C.make_params(6000, 5000, k, iters=10, seed=11, prec="fp64", core="pinv", trunc_rtol=trunc,
                      flags=C.FLAG_FOLLOW_ERR, err_samples=200000, err_seed=3)
    check_sketch(C, ctx, C.rbf_source(dev(X), dev(Y), sig), ref, p, 6000, 5000, err_ref)
    check_steps(C, ctx, ref, ref.P, ref.Q, k, 10)


def _midpoint_centres(X, pairs):
    return np.stack([(X[a] + X[b]) / 2.0 for a, b in pairs])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_snap_two_row_cluster_ties(ctx, C, prec):
    """Centres at the midpoints of row pairs (two-row clusters of equal
    weight): each must take the lower row of its pair whichever rounded
    distance is smaller, then the next centre at the same midpoint takes the
    other row; the oracle takes the same reading (tie window 1e-12 of
    d* + |z|^2 in FP64, 2^-16 in FP32)."""
    g = np.random.default_rng(77)
    M, d = 5000, 96
    X = g.standard_normal((M, d)) * 0.05
    rows = g.choice(M, 80, replace=False).tolist()
    pairs = [tuple(sorted(rows[2 * i:2 * i + 2])) for i in range(40)]
    # pull each (disjoint) pair close together so that it is the nearest pair to its midpoint
    for a, b in pairs:
        X[b] = X[a] + 1e-3 * g.standard_normal(d)
    if prec != "fp64":
        X = X.astype(np.float32).astype(np.float64)
    Z = _midpoint_centres(X, pairs)
    Z = np.concatenate([Z, Z[:10]])               # second centres at the same points
    dt = np.float64 if prec == "fp64" else np.float32
    Zd = Z.astype(dt)
    order, srt = C.cabs_snap(ctx, dev(X.astype(dt)), dev(Zd), prec=prec)
    tie = o.SNAP_TIE_RTOL if prec == "fp64" else 2.0 ** -16
    want_o, want_s = o.snap(X, Zd.astype(np.float64), tie_rtol=tie)
    assert to_np(order).tolist() == want_o.tolist()
    assert to_np(srt).tolist() == want_s.tolist()
    got = to_np(order).tolist()
    assert got[:40] == [a for a, _ in pairs]
    assert got[40:] == [b for _, b in pairs[:10]]


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_reduced_precision_excess_headline(ctx, C, dense_slice, prec):
    """The precision bar at the dense benchmark's k = 256 (stabilised core,
    truncation k 2^-24) on its slice: |err_mode / err_FP64 - 1| <= 1e-3, with
    the FP64 mode's error equal to the oracle's (checked above)."""
    A, Ad = dense_slice
    m, n = A.shape
    src = C.dense_source(Ad)
    errs = {}
    for pr in ("fp64", prec):
        p = C.make_params(m, n, 256, iters=5, seed=1607, prec=pr, core="stabilized", trunc_rtol=256 * U_FP32,
                          err_samples=0)
        sk = C.cabs_sketch(ctx, src, p)
        errs[pr] = float(to_np(sk.err)[0])
    assert abs(errs[prec] / errs["fp64"] - 1) <= 1e-3, errs
