"""Pins that tie the FP64 oracle to facts fixed by the paper or by mathematics.

Each ``pin_*`` takes the oracle function(s) it checks as arguments and raises
AssertionError when the fact does not hold, so the same pin runs against the
real oracle (tests/test_oracle_*.py) and against copies with a planted mistake
(tests/test_oracle_mutations.py), which it must reject.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from workloads import synth


# --------------------------------------------------------------- Philox / draw

def pin_philox_matches_numpy(philox_fn, cases=None):
    """numpy's Philox4x64-10 (an independent implementation) increments its
    256-bit counter before each block, so block(counter c) == numpy's first
    four raw outputs when started from counter c - 1."""
    rng = np.random.default_rng(5)
    if cases is None:
        cases = [((0, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (1607, 0)), ((0, 1, 0, 0), (2**64 - 1, 3)),
                 ((2**64 - 1, 7, 0, 0), (12345, 1)), ((0, 0, 0, 1), (99, 2))]
        for _ in range(20):
            cases.append((tuple(int(x) for x in rng.integers(0, 2**64, 4, dtype=np.uint64, endpoint=False)),
                          tuple(int(x) for x in rng.integers(0, 2**64, 2, dtype=np.uint64, endpoint=False))))
    for ctr, key in cases:
        c = ctr[0] | (ctr[1] << 64) | (ctr[2] << 128) | (ctr[3] << 192)
        c = (c - 1) % (1 << 256)
        start = np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
        want = tuple(int(x) for x in bg.random_raw(4))
        got = tuple(int(x) for x in philox_fn(ctr, key))
        assert got == want, (ctr, key)


def pin_draw_is_partial_fisher_yates(draw_fn, philox_fn, N=37, k=11, seed=3, tag=1):
    """The sparse-map draw equals Fisher-Yates run on an explicit array."""
    a = list(range(N))
    for i in range(k):
        r = philox_fn((i, 0, 0, 0), (seed, tag))[0]
        j = i + ((r * (N - i)) >> 64)
        a[i], a[j] = a[j], a[i]
    drawn, srt = draw_fn(seed, tag, N, k)
    assert list(drawn) == a[:k]
    assert list(srt) == sorted(a[:k])


def pin_draw_uniform(draw_fn, N=20, k=4, trials=3000, seed0=100):
    """Each index is drawn with probability k/N (chi-square), all distinct and in range."""
    counts = np.zeros(N)
    first = np.zeros(N)
    for s in range(trials):
        drawn, srt = draw_fn(seed0 + s, 0, N, k)
        assert len(set(drawn.tolist())) == k and drawn.min() >= 0 and drawn.max() < N
        assert np.all(np.diff(srt) > 0)
        counts[drawn] += 1
        first[drawn[0]] += 1
    from scipy.stats import chisquare
    assert chisquare(counts).pvalue > 1e-4
    assert chisquare(first).pvalue > 1e-4


# ----------------------------------------------------------------- sketching

def pin_gather_intersection(gather_fn, A, rows, cols):
    """W = R[:, J] = C[I, :] by definition (Algorithm 2, step 1)."""
    C, Rt, W = gather_fn(A, rows, cols)
    assert C.shape == (A.shape[0], len(cols)) and Rt.shape == (A.shape[1], len(rows))
    assert np.array_equal(W, C[rows, :])
    assert np.array_equal(W, Rt[cols, :].T)
    assert np.array_equal(C[:, 0], np.asarray(A[:, cols[0]], dtype=np.float64))
    assert np.array_equal(Rt[:, 0], np.asarray(A[rows[0], :], dtype=np.float64))


def pin_pinv_exact_recovery(gather_fn, sketch_fn, m=60, n=45, r=5, k=8, seed=11):
    """An exactly rank-r A with rank(W) = r is recovered exactly by C W^+ R."""
    A = synth.exact_lowrank_int(m, n, r, seed=seed)
    g = np.random.default_rng(seed)
    for _ in range(3):
        rows = np.sort(g.choice(m, k, replace=False))
        cols = np.sort(g.choice(n, k, replace=False))
        C, Rt, W = gather_fn(A, rows, cols)
        if np.linalg.matrix_rank(W) != r:
            continue
        sk = sketch_fn(C, Rt, W, m, n, "pinv", 0.0)
        assert sk.rank == r
        Ah = (sk.U * sk.S) @ sk.V.T
        assert np.linalg.norm(A - Ah) <= 1e-12 * np.linalg.norm(A)
        return
    raise AssertionError("no full-rank W drawn")


def pin_pinv_equals_pseudoskeleton(gather_fn, sketch_fn, m=50, n=40, k=9, seed=4):
    """U S V^T equals C W^+ R with W^+ from scipy's pinv (a different SVD driver)."""
    import scipy.linalg
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, n))
    rows = np.sort(g.choice(m, k, replace=False))
    cols = np.sort(g.choice(n, k, replace=False))
    C, Rt, W = gather_fn(A, rows, cols)
    sk = sketch_fn(C, Rt, W, m, n, "pinv", 0.0)
    want = C @ scipy.linalg.pinv(W) @ Rt.T
    got = (sk.U * sk.S) @ sk.V.T
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)


def pin_stabilized_rank1_closed_form(gather_fn, sketch_fn, m=40, n=30, k=6, seed=2):
    """For A = x y^T the stabilised routine returns exactly
    A * |x_I| |y_J| sqrt(mn) / (k |x| |y|): sigma_1 = |x_I||y_J|, N_c = |x||y_J|,
    N_r = |y||x_I|, S = sigma_1 sqrt(mn)/k. For sign vectors the factor is 1."""
    g = np.random.default_rng(seed)
    x = g.uniform(0.5, 2.0, m) * g.choice([-1.0, 1.0], m)
    y = g.uniform(0.5, 2.0, n) * g.choice([-1.0, 1.0], n)
    A = np.outer(x, y)
    rows = np.sort(g.choice(m, k, replace=False))
    cols = np.sort(g.choice(n, k, replace=False))
    C, Rt, W = gather_fn(A, rows, cols)
    sk = sketch_fn(C, Rt, W, m, n, "stabilized", 0.0)
    assert sk.rank == 1
    fac = np.linalg.norm(x[rows]) * np.linalg.norm(y[cols]) * math.sqrt(m * n) / (
        k * np.linalg.norm(x) * np.linalg.norm(y))
    Ah = (sk.U * sk.S) @ sk.V.T
    assert np.allclose(Ah, fac * A, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    assert abs(sk.S[0] - np.linalg.norm(x[rows]) * np.linalg.norm(y[cols]) * math.sqrt(m * n) / k) <= 1e-12 * sk.S[0]
    xs, ys = np.sign(x), np.sign(y)
    A = np.outer(xs, ys)
    C, Rt, W = gather_fn(A, rows, cols)
    sk = sketch_fn(C, Rt, W, m, n, "stabilized", 0.0)
    assert np.allclose((sk.U * sk.S) @ sk.V.T, A, rtol=0, atol=1e-12)


def pin_stabilized_rank2_hadamard(gather_fn, sketch_fn):
    """A = a x1 y1^T + b x2 y2^T with Hadamard sign vectors whose samples stay
    orthogonal: W's SVD is known in closed form and the stabilised routine
    recovers A exactly, with S = (a sqrt(mn), b sqrt(mn))."""
    H8 = np.array([[1, 1, 1, 1, 1, 1, 1, 1], [1, -1, 1, -1, 1, -1, 1, -1],
                   [1, 1, -1, -1, 1, 1, -1, -1], [1, -1, -1, 1, 1, -1, -1, 1]], dtype=np.float64)
    x1, x2 = np.tile(H8[1], 2), np.tile(H8[2], 2)          # m = 16
    y1, y2 = np.tile(H8[1], 3), np.tile(H8[3], 3)          # n = 24
    a, b = 3.0, 0.5
    A = a * np.outer(x1, y1) + b * np.outer(x2, y2)
    rows = np.array([0, 1, 2, 3])      # x1 = (1,-1,1,-1), x2 = (1,1,-1,-1): orthogonal
    cols = np.array([8, 9, 10, 11])    # y1 = (1,-1,1,-1), y2 = (1,-1,-1,1): orthogonal
    C, Rt, W = gather_fn(A, rows, cols)
    sk = sketch_fn(C, Rt, W, 16, 24, "stabilized", 0.0)
    assert sk.rank == 2
    assert np.allclose(sk.sig[:2], [a * 4, b * 4], rtol=1e-14)
    assert np.allclose(sk.S[:2], [a * math.sqrt(16 * 24), b * math.sqrt(16 * 24)], rtol=1e-13)
    assert np.allclose((sk.U * sk.S) @ sk.V.T, A, atol=1e-12)


def pin_unit_columns_and_truncation(gather_fn, sketch_fn, m=70, n=50, k=10, r=4, seed=9):
    """Kept columns of U and V have unit norm, dropped ones are zero, and a
    rank-r W keeps exactly r components; singular values match scipy's gesvd."""
    import scipy.linalg
    A = synth.exact_lowrank_int(m, n, r, seed=seed) + 0.0
    g = np.random.default_rng(seed)
    rows = np.sort(g.choice(m, k, replace=False))
    cols = np.sort(g.choice(n, k, replace=False))
    C, Rt, W = gather_fn(A, rows, cols)
    for mode in ("pinv", "stabilized"):
        sk = sketch_fn(C, Rt, W, m, n, mode, 0.0)
        assert sk.rank == np.linalg.matrix_rank(W)
        nu = np.linalg.norm(sk.U, axis=0)
        nv = np.linalg.norm(sk.V, axis=0)
        assert np.allclose(nu[:sk.rank], 1, atol=1e-14) and np.all(nu[sk.rank:] == 0)
        assert np.allclose(nv[:sk.rank], 1, atol=1e-14) and np.all(nv[sk.rank:] == 0)
        assert np.all(sk.S[sk.rank:] == 0) and np.all(sk.S[:sk.rank] > 0)
        ref = scipy.linalg.svd(W, compute_uv=False, lapack_driver="gesvd")
        assert np.allclose(sk.sig, ref, rtol=1e-12, atol=1e-12 * ref[0])


# ------------------------------------------------------------------- k-means

def _blobs(m, k2, d=2, seed=0, spread=0.05):
    g = np.random.default_rng(seed)
    centers = g.uniform(-5, 5, (k2, d))
    lab = np.arange(m) % k2
    return centers[lab] + spread * g.standard_normal((m, d))


def pin_kmeans_bruteforce_optimum(kmeans_fn, trials=6):
    """On tiny well-separated blobs, Lloyd from one point per blob reaches the
    weighted-SSE optimum found by enumerating every labelling."""
    for t in range(trials):
        m, k2 = (7, 2) if t % 2 == 0 else (8, 3)
        X = _blobs(m, k2, seed=t)
        p = [0.0, 1.0, 2.0][t % 3]
        w = np.linalg.norm(X, axis=1) ** p if p else np.ones(m)
        best = np.inf
        for lab in itertools.product(range(k2), repeat=m):
            lab = np.array(lab)
            e = 0.0
            for j in range(k2):
                mem = lab == j
                if mem.any():
                    z = (w[mem, None] * X[mem]).sum(0) / w[mem].sum()
                    e += float((w[mem] * ((X[mem] - z) ** 2).sum(1)).sum())
            best = min(best, e)
        init = [j for j in range(k2)]          # rows 0..k2-1 lie in distinct blobs
        res = kmeans_fn(X, init, 4, p)
        D = np.array([((X - z) ** 2).sum(1) for z in res.Z]).T
        e_final = float((w * D.min(1)).sum())
        assert e_final <= best * (1 + 1e-9) + 1e-12, (e_final, best)


def pin_kmeans_steps_exhaustive(kmeans_fn, M=40, d=3, k2=5, iters=4, p=1.0, seed=3):
    """Every assignment is the lowest-index minimum over all centres, every
    centre is the weighted mean of its members (or unchanged when empty), and
    the weighted objective never increases (Eq. wkmeans)."""
    g = np.random.default_rng(seed)
    X = g.standard_normal((M, d))
    res = kmeans_fn(X, list(range(k2)), iters, p)
    w = [math.sqrt(sum(float(v) ** 2 for v in X[l])) ** p for l in range(M)]
    for t in range(iters):
        Z = res.centres[t]
        for l in range(M):
            ds = [sum((float(X[l, q]) - float(Z[j, q])) ** 2 for q in range(d)) for j in range(k2)]
            jbest = min(range(k2), key=lambda j: (ds[j], j))
            assert res.labels[t][l] == jbest
        Zn = res.centres[t + 1]
        for j in range(k2):
            mem = [l for l in range(M) if res.labels[t][l] == j]
            ws = sum(w[l] for l in mem)
            if ws > 0:
                want = [sum(w[l] * float(X[l, q]) for l in mem) / ws for q in range(d)]
            else:
                want = list(Z[j])
            assert np.allclose(Zn[j], want, rtol=1e-13, atol=1e-13)
        e = sum(w[l] * sum((float(X[l, q]) - float(Z[res.labels[t][l], q])) ** 2 for q in range(d)) for l in range(M))
        assert abs(e - res.energy[t]) <= 1e-10 * max(1.0, e)
    assert all(res.energy[t + 1] <= res.energy[t] * (1 + 1e-12) for t in range(iters - 1))


def pin_kmeans_ties_and_empty(kmeans_fn):
    """A point equidistant from two centres goes to the lower index; a centre
    that wins no point keeps its position."""
    X = np.array([[0.0, 0.0], [2.0, 0.0], [1.0, 0.0], [10.0, 10.0]])
    res = kmeans_fn(X, [0, 1], 1, 0.0)
    assert res.labels[0].tolist() == [0, 1, 0, 1]
    X = np.array([[1.0, 1.0], [1.0, 1.0], [1.5, 1.0], [5.0, 5.0]])
    res = kmeans_fn(X, [0, 1, 3], 2, 0.0)
    # centre 1 duplicates centre 0 and loses every tie -> empty, keeps (1, 1)
    assert res.labels[0].tolist() == [0, 0, 0, 2]
    assert np.array_equal(res.centres[1][1], [1.0, 1.0])
    assert np.allclose(res.centres[1][0], [3.5 / 3, 1.0])


def pin_kmeans_matches_sklearn(kmeans_fn, M=300, d=6, k2=7, iters=5, seed=1):
    """sklearn's weighted Lloyd (independent code) gives the same centres
    when no cluster empties."""
    import pytest
    sk = pytest.importorskip("sklearn.cluster")
    g = np.random.default_rng(seed)
    X = _blobs(M, k2, d=d, seed=seed, spread=1.0)
    w = np.linalg.norm(X, axis=1) ** 1.5
    init = list(range(k2))
    res = kmeans_fn(X, init, iters, 1.5)
    km = sk.KMeans(n_clusters=k2, init=X[init], n_init=1, max_iter=iters, tol=0.0,
                   algorithm="lloyd").fit(X, sample_weight=w)
    assert np.allclose(km.cluster_centers_, res.Z, rtol=1e-10, atol=1e-10)


def pin_snap_bruteforce(snap_fn, M=30, d=3, k2=6, seed=8):
    """Greedy distinct nearest rows, checked with explicit loops; the result is sorted."""
    g = np.random.default_rng(seed)
    X = g.standard_normal((M, d))
    Z = g.standard_normal((k2, d)) * 0.3
    Z[1] = Z[0]                      # two centres with the same nearest row
    order, srt = snap_fn(X, Z)
    taken = []
    for j in range(k2):
        ds = [(sum((float(X[l, q]) - float(Z[j, q])) ** 2 for q in range(d)), l) for l in range(M) if l not in taken]
        best = min(ds)
        zz = sum(float(Z[j, q]) ** 2 for q in range(d))
        # rows within the tie window of the nearest; these inputs have none
        assert [l for v, l in ds if v <= best[0] + 1e-12 * (best[0] + zz)] == [best[1]]
        taken.append(best[1])
    assert order.tolist() == taken
    assert srt.tolist() == sorted(taken)
    assert len(set(taken)) == k2


def _midpoint_case(flip, d=7, seed=21, offset=0.0, spread=1.0):
    """Rows a < b of a random X (offset + spread N(0, 1) entries) and their
    midpoint z = (x_a + x_b) / 2, found so that the FP64 squared distances by
    direct differences (summed in dimension order) come out unequal: with
    flip, the higher row b looks strictly nearer, otherwise a does.
    Mathematically |x_a - z| = |x_b - z|."""
    g = np.random.default_rng(seed)
    for _ in range(10000):
        X = offset + spread * g.standard_normal((12, d))
        a, b = sorted(g.choice(12, 2, replace=False).tolist())
        z = (X[a] + X[b]) / 2.0
        da = sum((float(X[a, q]) - float(z[q])) ** 2 for q in range(d))
        db = sum((float(X[b, q]) - float(z[q])) ** 2 for q in range(d))
        others = [sum((float(X[l, q]) - float(z[q])) ** 2 for q in range(d)) for l in range(12) if l not in (a, b)]
        if min(others) > 2 * max(da, db) and ((db < da) if flip else (da < db)):
            return X, z, a, b
    raise AssertionError("no rounding-split midpoint found")


def pin_snap_midpoint_tie(snap_fn):
    """Section 3.2 replaces a centre by its closest in-sample point; the
    centre of a two-row cluster is the midpoint of the rows, equidistant
    from both, so the tie goes to the lower row whichever rounded distance is
    smaller. A genuine difference of 1e-9 relative (far above FP64 rounding,
    far below any data scale) is not a tie: the nearer row wins even when its
    index is higher."""
    for flip in (False, True):
        X, z, a, b = _midpoint_case(flip)
        order, _ = snap_fn(X, z[None, :])
        assert order.tolist() == [a], (flip, order, a, b)
        # a second centre at the same point takes the other row
        order, srt = snap_fn(X, np.stack([z, z]))
        assert order.tolist() == [a, b]
    # far from the origin, rounding of x - z scales with |z|, not |x - z|:
    # the window must be relative to d* + |z|^2
    X, z, a, b = _midpoint_case(True, offset=1000.0, spread=1e-3)
    order, _ = snap_fn(X, z[None, :])
    assert order.tolist() == [a]
    X, z, a, b = _midpoint_case(False)
    u = (X[b] - X[a]) / np.linalg.norm(X[b] - X[a])
    # moving z by e towards x_b lowers |x_b - z|^2 - |x_a - z|^2 by 4 e |x_b - x_a| / 2
    e = 1e-9 * (float(((X[a] - z) ** 2).sum()) + float((z * z).sum())) / (2.0 * np.linalg.norm(X[b] - X[a]))
    order, _ = snap_fn(X, (z + e * u)[None, :])
    assert order.tolist() == [b]


# ------------------------------------------------------------ hard threshold

def pin_threshold_bruteforce(thr_fn, M=40, d=5, k2=9, seed=12):
    """The k2 rows of largest norm, found by repeated maximum extraction with
    explicit loops (ties to the lower index); the result is sorted."""
    g = np.random.default_rng(seed)
    X = g.standard_normal((M, d)) * g.uniform(0.2, 3.0, size=(M, 1))
    X[7] = -X[3]          # equal norms: row 3 wins the tie if both are near the cut
    left = list(range(M))
    pick = []
    for _ in range(k2):
        best = None
        for l in left:
            v = sum(float(X[l, q]) ** 2 for q in range(d))
            if best is None or v > best[0]:
                best = (v, l)
        pick.append(best[1])
        left.remove(best[1])
    assert thr_fn(X, k2).tolist() == sorted(pick)


def pin_threshold_known_scales(thr_fn):
    """Rows c_l u for a fixed unit vector u: the top k2 are the rows with the
    largest |c_l| (signs do not matter); equal |c_l| resolve to the lower row."""
    u = np.array([0.6, 0.0, 0.8])
    c = np.array([1.0, -5.0, 2.0, 5.0, -0.5, 3.0, 3.0, 0.1])
    X = c[:, None] * u[None, :]
    assert thr_fn(X, 1).tolist() == [1]           # |-5| == |5|: the lower row
    assert thr_fn(X, 2).tolist() == [1, 3]
    assert thr_fn(X, 3).tolist() == [1, 3, 5]     # 3 ties with row 6: the lower row
    assert thr_fn(X, 5).tolist() == [1, 2, 3, 5, 6]
    assert thr_fn(X, 8).tolist() == list(range(8))
    assert thr_fn(np.ones((5, 2)), 2).tolist() == [0, 1]   # all equal: the first rows


# --------------------------------------------------------- orthogonalisation

def pin_orthogonalize(orth_fn, m=60, n=45, r=6, seed=13):
    """The SVD form of U diag(S) V^T: the same matrix, orthonormal factors,
    and the singular values of the explicit product (numpy's SVD of the dense
    m x n matrix, an independent route); dropped directions of an exactly
    rank-deficient sketch; a closed form with orthogonal inputs."""
    g = np.random.default_rng(seed)
    U = g.standard_normal((m, r))
    V = g.standard_normal((n, r))
    S = np.abs(g.standard_normal(r)) + 0.5
    X, s, Y = orth_fn(U, S, V)
    A = (U * S) @ V.T
    assert np.allclose((X * s) @ Y.T, A, atol=1e-12 * np.abs(A).max())
    assert np.allclose(X.T @ X, np.eye(len(s)), atol=1e-12)
    assert np.allclose(Y.T @ Y, np.eye(len(s)), atol=1e-12)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False)[:r], rtol=1e-12)
    assert np.all(np.diff(s) <= 0)
    # two equal columns of U: the rank drops to r - 1
    U2 = U.copy()
    U2[:, 1] = U2[:, 0]
    X2, s2, Y2 = orth_fn(U2, S, V)
    assert len(s2) == r - 1
    assert np.allclose((X2 * s2) @ Y2.T, (U2 * S) @ V.T, atol=1e-12 * np.abs(A).max())
    # orthonormal U and V already: s is S sorted, up to signs of the columns
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    X3, s3, Y3 = orth_fn(Qu, S, Qv)
    assert np.allclose(s3, np.sort(S)[::-1], rtol=1e-13)


# ------------------------------------------------------------ BR-CUR, Sketch-CUR

def pin_embed(embed_fn, sketching_fn, gather_fn):
    """Algorithm 2, step 2: P = U S^(1/2). Closed form: orthonormal U with
    S = (4, 9, 0) gives P = U diag(2, 3, 0). Identity: the pseudo-skeleton
    core has U diag(S) V^T = C W^+ R (Section 2.2, Eq. W), so the two
    embeddings satisfy P Q^T = C W^+ R, here against an LU solve for W^-1
    on an exactly rank-3 matrix with rank(W) = 3, whose P Q^T is A itself."""
    g = np.random.default_rng(17)
    U, _ = np.linalg.qr(g.standard_normal((6, 3)))
    P = embed_fn(U, np.array([4.0, 9.0, 0.0]))
    assert np.allclose(P, U * np.array([2.0, 3.0, 0.0]), rtol=0, atol=1e-15)
    A = synth.exact_lowrank_int(40, 30, 3, seed=5)
    rows, cols = np.array([2, 11, 29]), np.array([0, 7, 21])
    C, Rt, W = gather_fn(A, rows, cols)
    assert np.linalg.matrix_rank(W) == 3
    sk = sketching_fn(C, Rt, W, 40, 30, "pinv")
    Pm, Qm = embed_fn(sk.U, sk.S), embed_fn(sk.V, sk.S)
    want = C @ np.linalg.solve(W, Rt.T)
    assert np.linalg.norm(Pm @ Qm.T - want) <= 1e-10 * np.linalg.norm(want)
    assert np.linalg.norm(Pm @ Qm.T - A) <= 1e-10 * np.linalg.norm(A)


def pin_pinv_trunc(pinv_fn):
    """Closed forms on matrices with known singular values. 5 x 3 with
    s = (1, 1e-3, 3e-8): the floor 5 x 2^-52 = 1.1e-15 keeps all three (its
    square root, 3.3e-8, would drop the third); 50 x 3 with
    s = (1, 1e-3, 3e-15): the floor 50 x 2^-52 = 1.1e-14 drops the third
    (3 x 2^-52 = 6.7e-16, from the smaller dimension, would keep it); a
    tolerance of 1e-2 keeps the first only."""
    g = np.random.default_rng(3)
    Q1, _ = np.linalg.qr(g.standard_normal((5, 3)))
    Q2, _ = np.linalg.qr(g.standard_normal((3, 3)))
    s = np.array([1.0, 1e-3, 3e-8])
    B = (Q1 * s) @ Q2.T
    want = (Q2 / s) @ Q1.T
    assert np.linalg.norm(pinv_fn(B) - want) <= 1e-6 * np.linalg.norm(want)
    want_t = (Q2[:, :1] / s[:1]) @ Q1[:, :1].T
    assert np.allclose(pinv_fn(B, 1e-2), want_t, rtol=0, atol=1e-12)
    Q3, _ = np.linalg.qr(g.standard_normal((50, 3)))
    s2 = np.array([1.0, 1e-3, 3e-15])
    B2 = (Q3 * s2) @ Q2.T
    want2 = (Q2[:, :2] / s2[:2]) @ Q3[:, :2].T
    assert np.allclose(pinv_fn(B2), want2, rtol=0, atol=1e-9)
    # full rank square: the inverse (LU, an independent routine)
    W = g.standard_normal((6, 6)) + 3 * np.eye(6)
    assert np.allclose(pinv_fn(W), np.linalg.solve(W, np.eye(6)), atol=1e-12)
    assert np.all(pinv_fn(np.zeros((4, 3))) == 0) and pinv_fn(np.zeros((4, 3))).shape == (3, 4)


def pin_br_cur(br_cur_fn, source_cls):
    """Algorithm 1 on facts the mathematics fixes: (1) an exactly rank-4
    matrix is recovered exactly from 6 base and 10 target rows and columns;
    (2) with the target equal to the base, U* = W^-1 (the pseudo-skeleton
    C W^+ R of Eq. W; Nystrom for a symmetric PSD A with equal rows and
    columns), checked against an LU solve; (3) U* satisfies the normal
    equations C_bar^T (M - C_bar U* R_bar) R_bar^T = 0 of step 4."""
    from workloads import synth
    g = np.random.default_rng(5)
    A = synth.exact_lowrank_int(60, 50, 4, seed=9)
    rb = np.sort(g.choice(60, 6, replace=False))
    cb = np.sort(g.choice(50, 6, replace=False))
    rt = np.sort(g.choice(60, 10, replace=False))
    ct = np.sort(g.choice(50, 10, replace=False))
    r = br_cur_fn(source_cls(A), rb, cb, rt, ct)
    assert r.C.shape == (60, 6) and r.U.shape == (6, 6) and r.Rt.shape == (50, 6)
    assert np.allclose(r.C @ r.U @ r.Rt.T, A, atol=1e-9 * np.abs(A).max())
    # (2) target = base, full-rank W
    B = g.standard_normal((40, 30))
    rows = np.sort(g.choice(40, 7, replace=False))
    cols = np.sort(g.choice(30, 7, replace=False))
    r2 = br_cur_fn(source_cls(B), rows, cols, rows, cols)
    W = B[np.ix_(rows, cols)]
    assert np.allclose(r2.U, np.linalg.solve(W, np.eye(7)), atol=1e-10)
    assert np.allclose(r2.C, B[:, cols]) and np.allclose(r2.Rt, B[rows, :].T)
    # symmetric PSD, same rows and columns: Nystrom C W^-1 C^T
    G = g.standard_normal((30, 30))
    K = G @ G.T
    idx = np.sort(g.choice(30, 8, replace=False))
    r3 = br_cur_fn(source_cls(K), idx, idx, idx, idx)
    Cn = K[:, idx]
    assert np.allclose(r3.C @ r3.U @ r3.Rt.T, Cn @ np.linalg.solve(K[np.ix_(idx, idx)], Cn.T),
                       atol=1e-8 * np.abs(K).max())
    # (3) normal equations, independent target
    rt4 = np.sort(g.choice(40, 15, replace=False))
    ct4 = np.sort(g.choice(30, 12, replace=False))
    r4 = br_cur_fn(source_cls(B), rows, cols, rt4, ct4)
    Cbar = B[np.ix_(rt4, cols)]
    Rbar = B[np.ix_(rows, ct4)]
    M = B[np.ix_(rt4, ct4)]
    grad = Cbar.T @ (M - Cbar @ r4.U @ Rbar) @ Rbar.T
    assert np.abs(grad).max() < 1e-9 * np.abs(M).max() * np.abs(Cbar).max() * np.abs(Rbar).max()


# ------------------------------------------------------ leverage-score follow-up

def pin_leverage_scores(lev_fn, orth_fn):
    """Leverage scores of the pilot form P Q^T through its SVD form equal the
    diagonal of the hat matrix P (P^T P)^-1 P^T (an LU solve, independent of
    any SVD) for full-rank factors, and sum to the rank."""
    g = np.random.default_rng(21)
    P = g.standard_normal((80, 6))
    Q = g.standard_normal((50, 6))
    X, _, Y = orth_fn(P, np.ones(6), Q)
    hat = np.einsum("ij,ji->i", P, np.linalg.solve(P.T @ P, P.T))
    assert np.allclose(lev_fn(X), hat, atol=1e-12)
    hat_q = np.einsum("ij,ji->i", Q, np.linalg.solve(Q.T @ Q, Q.T))
    assert np.allclose(lev_fn(Y), hat_q, atol=1e-12)
    assert abs(lev_fn(X).sum() - 6) < 1e-12


def pin_weighted_sample(ws_fn):
    """A-Res sampling: (1) k = N selects everything; (2) zero weights are
    never drawn while positive ones remain; (3) over 4000 seeds the inclusion
    frequency of each index for k = 2 matches the closed form of successive
    weighted draws without replacement, P(i in S) = p_i + sum_{j != i} p_j
    p_i / (1 - p_j), within 4.5 standard errors; (4) equal weights reduce to
    the k smallest -ln u, i.e. the k largest u."""
    w = np.array([5.0, 1.0, 0.0, 2.0, 2.0])
    assert ws_fn(w, 5, 1, 6)[0].tolist() == [0, 1, 2, 3, 4]
    for seed in range(50):
        sel = ws_fn(w, 4, seed, 6)[0].tolist()
        assert 2 not in sel and sorted(sel) == sel and len(set(sel)) == 4
    p = w / w.sum()
    want = np.array([p[i] + sum(p[j] * p[i] / (1 - p[j]) for j in range(5) if j != i) for i in range(5)])
    T = 4000
    cnt = np.zeros(5)
    for seed in range(T):
        cnt[ws_fn(w, 2, seed, 7)[0]] += 1
    freq = cnt / T
    se = np.sqrt(np.maximum(want * (1 - want), 1e-12) / T)
    assert np.all(np.abs(freq - want) <= 4.5 * se + 1e-12), (freq, want)
    u = philox_uniform_for_pin(11, 6, 9)
    assert ws_fn(np.ones(9), 3, 11, 6)[0].tolist() == sorted(np.argsort(-u, kind="stable")[:3].tolist())


def philox_uniform_for_pin(seed, tag, N):
    """Uniforms from numpy's own Philox4x64-10 (an independent implementation
    of the generator; it increments its counter before each block): word 0 of
    block (i, 0, 0, 0), mapped to ((r >> 11) + 1/2) 2^-53."""
    out = []
    for i in range(N):
        c = (i - 1) % (1 << 256)
        start = np.array([(c >> (64 * t)) & (2**64 - 1) for t in range(4)], dtype=np.uint64)
        bg = np.random.Philox(key=np.array([seed, tag], dtype=np.uint64), counter=start)
        r = int(bg.random_raw(4)[0])
        out.append(((r >> 11) + 0.5) * 2.0 ** -53)
    return np.array(out)


# ---------------------------------------------------------------------- error

def pin_error_closed_form(err_fn):
    """|A - U S V^T|_F / |A|_F on a case computed by hand: A = I_2, U = V = e1, S = 1
    leaves the residual e2 e2^T, so the error is 1/sqrt(2)."""
    A = np.eye(2)
    U = np.array([[1.0], [0.0]])
    V = np.array([[1.0], [0.0]])
    assert abs(err_fn(A, U, np.array([1.0]), V) - 1 / math.sqrt(2)) < 1e-15
    assert err_fn(A, np.eye(2), np.ones(2), np.eye(2)) == 0.0


def pin_sampled_error_closed_form(err_fn, source_cls):
    """The sampled error on a case computed by hand: A = u v^T with distinct
    entries, approximated by U S V^T = A / 2 (U = u/|u|, V = v/|v|,
    S = |u||v| / 2). Every entry then has a - a_hat = a / 2, so the error is
    1/2 whatever entries are drawn; with S = |u||v| it is 0."""
    u = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    v = np.array([1.0, -2.0, 0.5, 3.0, 7.0])
    src = source_cls(np.outer(u, v))
    U = (u / np.linalg.norm(u))[:, None]
    V = (v / np.linalg.norm(v))[:, None]
    S = np.array([np.linalg.norm(u) * np.linalg.norm(v) / 2])
    assert abs(err_fn(src, U, S, V, 5, 400) - 0.5) < 1e-14
    assert err_fn(src, U, 2 * S, V, 5, 400) < 1e-14


# ---------------------------------------------------------------- RBF entries

def pin_rbf_closed_forms(entries_fn):
    """exp(-|x - y|^2 / (2 sigma^2)) at points chosen by hand: x = y gives 1;
    sigma = 1 with |x - y|^2 = 2 gives exp(-1), with |x - y|^2 = 4 (an L1
    distance of 2) exp(-2); sigma = 2 with |x - y|^2 = 8 gives exp(-1)."""
    X = np.array([[0.0, 0.0], [1.0, 1.0]], dtype=np.float32)
    Y = np.array([[0.0, 0.0], [0.0, 2.0]], dtype=np.float32)
    v = entries_fn(X, Y, 1.0, [0, 1, 0], [0, 0, 1])
    assert v[0] == 1.0 and abs(v[1] - np.exp(-1.0)) < 1e-16 and abs(v[2] - np.exp(-2.0)) < 1e-16
    w = entries_fn(np.array([[2.0, 2.0]], dtype=np.float32), np.zeros((1, 2), dtype=np.float32), 2.0, [0], [0])
    assert abs(w[0] - np.exp(-1.0)) < 1e-16


def pin_rbf_block_and_gather(block_fn, gather_fn, entries_fn, m=9, n=7, d=3, seed=31):
    """Every generated entry is the kernel of its own pair: block[a, b] =
    entry(rows[a], cols[b]); the gather's C = A[:, cols], R^T = A[rows, :]^T
    and W = A[rows, cols] of the same implicit matrix."""
    g = np.random.default_rng(seed)
    X = g.standard_normal((m, d)).astype(np.float32)
    Y = g.standard_normal((n, d)).astype(np.float32)
    sigma = 1.3
    rows, cols = np.array([8, 0, 5]), np.array([6, 2])
    def A(ii, jj):
        I, J = np.meshgrid(ii, jj, indexing="ij")
        return entries_fn(X, Y, sigma, I.ravel(), J.ravel()).reshape(I.shape)
    assert np.allclose(block_fn(X, Y, sigma, rows, cols), A(rows, cols), rtol=1e-15, atol=0)
    C, Rt, W = gather_fn(X, Y, sigma, rows, cols)
    assert np.allclose(C, A(np.arange(m), cols), rtol=1e-15, atol=0)
    assert np.allclose(Rt, A(rows, np.arange(n)).T, rtol=1e-15, atol=0)
    assert np.allclose(W, A(rows, cols), rtol=1e-15, atol=0)


# ---------------------------------------------------- weights, encoding error

def pin_upsilon_weights(ups_fn):
    """Upsilon(|x|) = |x|^p on rows of norm 5 and 0: p = 1 gives 5 and 0, p = 2
    gives 25 and 0, p = 0 gives 1 for both (0^0 = 1)."""
    X = np.array([[3.0, 4.0], [0.0, 0.0]])
    assert ups_fn(X, 1.0).tolist() == [5.0, 0.0]
    assert ups_fn(X, 2.0).tolist() == [25.0, 0.0]
    assert ups_fn(X, 0.0).tolist() == [1.0, 1.0]


def pin_encoding_error_closed_form(enc_fn):
    """Points 0, 1, 3, 10 on a line with representatives rows 0 and 3 (the
    points 0 and 10): nearest squared distances 0, 1, 9, 0, labels 0, 0, 0, 1,
    largest cluster 3; the unweighted error is 10, and with Upsilon(t) = t
    (weights 0, 1, 3, 10) it is 1 + 27 = 28."""
    X = np.array([[0.0], [1.0], [3.0], [10.0]])
    err, lab, T = enc_fn(X, [0, 3], 0.0)
    assert err == 10.0 and lab.tolist() == [0, 0, 0, 1] and T == 3
    assert enc_fn(X, [0, 3], 1.0)[0] == 28.0


# ------------------------------------------------------- the Algorithm 2 driver

def pin_follow_up_improves_encoding(cabs_fn, source_cls, trials=20):
    """Step 3 of Algorithm 2 moves the representatives from the pilot draw to
    the snapped k-means centres, which lowers the weighted encoding error of
    both embeddings (the premise of Theorem 2, e_f < e_p) on at least 95 % of
    seeds of a decaying-spectrum matrix (strictly: the k-means iterations
    move the centres)."""
    A, _, _, _ = synth.decaying_lowrank_host(300, 240, rank=40, decay=10, noise_std=1e-4,
                                             seed=3, dtype=np.float64)
    src = source_cls(A)
    ok = 0
    for seed in range(trials):
        r = cabs_fn(src, 16, iters=5, seed=seed, mode="stabilized")
        ok += (r.e_follow[0] < r.e_pilot[0]) and (r.e_follow[1] < r.e_pilot[1])
    assert ok >= 0.95 * trials


def pin_driver_wiring(cabs_fn, source_cls, sketch_fn, embed_fn, kmeans_fn, snap_fn):
    """Algorithm 2 composes its steps in order: P = U S^(1/2), Q = V S^(1/2) of
    the pilot sketch (step 2); k-means on P and Q from the first k2 pilot
    draws, snapped (step 3); the final sketch is the sketching routine on the
    gather at the snapped indices (step 4), which here differ from the pilot
    ones."""
    A = synth.plain_lowrank(120, 90, 6)
    src = source_cls(A)
    r = cabs_fn(src, 10, k2=7, iters=3, seed=5, mode="stabilized")
    assert np.array_equal(r.P, embed_fn(r.pilot.U, r.pilot.S))
    assert np.array_equal(r.Q, embed_fn(r.pilot.V, r.pilot.S))
    km_r = kmeans_fn(r.P, r.pilot_rows_drawn[:7], 3)
    km_c = kmeans_fn(r.Q, r.pilot_cols_drawn[:7], 3)
    assert np.array_equal(r.rows, snap_fn(r.P, km_r.Z)[1]) and np.array_equal(r.cols, snap_fn(r.Q, km_c.Z)[1])
    assert not (np.array_equal(r.rows, r.pilot_rows[:7]) and np.array_equal(r.cols, r.pilot_cols[:7]))
    f = sketch_fn(*src.gather(r.rows, r.cols), 120, 90, "stabilized")
    assert np.array_equal(r.final.U, f.U) and np.array_equal(r.final.S, f.S) and np.array_equal(r.final.V, f.V)


# ----------------------------------------------- uniforms and sampled entries

def _numpy_philox_words(seed, tag, t):
    """The four words of block (t, 0, 0, 0) under key (seed, tag), from numpy's
    own Philox4x64-10 (it increments its counter before each block)."""
    c = (t - 1) % (1 << 256)
    start = np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array([seed, tag], dtype=np.uint64), counter=start)
    return [int(x) for x in bg.random_raw(4)]


def pin_philox_uniform(pu_fn, seed=11, tag=6, N=9):
    """u_i = ((r_i >> 11) + 1/2) 2^-53 from word 0 of numpy's Philox block i:
    every u lies in (0, 1), 2^53 u - 1/2 is a whole number, and the values are
    those of the independent generator."""
    u = pu_fn(seed, tag, N)
    assert np.array_equal(u, philox_uniform_for_pin(seed, tag, N))
    assert np.all((u > 0) & (u < 1))
    x = u * 2.0 ** 53 - 0.5
    assert np.array_equal(x, np.floor(x))


def pin_eval_samples(es_fn, seed=5, m=1000, n=777, count=12):
    """The sampled error's entries: row hi64(w0 m), column hi64(w1 n) of
    block (t, 0, 0, 0) under key (seed, 2), the words from numpy's Philox."""
    ii, jj = es_fn(seed, m, n, count)
    for t in range(count):
        w = _numpy_philox_words(seed, 2, t)
        assert ii[t] == (w[0] * m) >> 64 and jj[t] == (w[1] * n) >> 64, t


def pin_sq_dists(sq_fn):
    """Squared distances by hand: from (1, 1) the points (0, 0), (3, 4) and
    (1, 1) lie at 2, 13 and 0."""
    X = np.array([[0.0, 0.0], [3.0, 4.0], [1.0, 1.0]])
    assert sq_fn(X, np.array([1.0, 1.0])).tolist() == [2.0, 13.0, 0.0]


def pin_csr_gather(csr_cls, dense_cls):
    """The sparse source's gathers and entries equal the dense source's on the
    same matrix held densely (numpy indexing of a dense array, independent of
    scipy's sparse slicing), bit for bit; rows with no stored entries gather
    as zeros."""
    ip, ix, v = synth.sparse_lowrank(300, 200, 0.03, rank=4, seed=3)
    src = csr_cls(ip, ix, v, 200)
    A = np.zeros((300, 200))
    for r in range(300):
        A[r, ix[ip[r]:ip[r + 1]]] = v[ip[r]:ip[r + 1]]
    dense = dense_cls(A)
    g = np.random.default_rng(2)
    rows = np.sort(g.choice(300, 17, replace=False))
    cols = np.sort(g.choice(200, 13, replace=False))
    for a, b in zip(src.gather(rows, cols), dense.gather(rows, cols)):
        assert a.shape == b.shape and np.array_equal(a, b)
    ii, jj = g.integers(0, 300, 500), g.integers(0, 200, 500)
    assert np.array_equal(src.entries(ii, jj), dense.entries(ii, jj))
