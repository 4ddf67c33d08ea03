"""The FP64 oracle checked against what the paper and mathematics fix (no GPU)."""
import numpy as np
import pytest

from oracle import cabs_ref as o
from tests import oracle_pins as pins
from workloads import synth


def test_philox_matches_numpy_philox():
    pins.pin_philox_matches_numpy(o.philox4x64_10)


def test_philox_vectorised_matches_scalar():
    g = np.random.default_rng(0)
    c = g.integers(0, 2**63, (4, 64), dtype=np.int64).astype(np.uint64) * np.uint64(2)
    key = (2**64 - 5, 77)
    v = o.philox4x64_10_vec(c[0], c[1], c[2], c[3], *key)
    for t in range(64):
        want = o.philox4x64_10(tuple(int(x) for x in c[:, t]), key)
        assert tuple(int(x[t]) for x in v) == want


def test_mulhi64():
    assert o.mulhi64(2**63, 10) == 5
    assert o.mulhi64(2**64 - 1, 2**64 - 1) == 2**64 - 2
    a = np.array([2**63, 2**64 - 1, 12345], dtype=np.uint64)
    assert o.mulhi64_vec(a, 1000).tolist() == [500, 999, 0]


def test_draw_is_partial_fisher_yates():
    pins.pin_draw_is_partial_fisher_yates(o.draw_indices, o.philox4x64_10)
    pins.pin_draw_is_partial_fisher_yates(o.draw_indices, o.philox4x64_10, N=5, k=5, seed=9, tag=0)


def test_draw_uniform_distinct_sorted():
    pins.pin_draw_uniform(o.draw_indices)


def test_draw_full_permutation_and_edges():
    d, s = o.draw_indices(4, 0, 16, 16)
    assert sorted(d.tolist()) == list(range(16)) and s.tolist() == list(range(16))
    d, s = o.draw_indices(4, 0, 1, 1)
    assert d.tolist() == [0]
    d, s = o.draw_indices(4, 0, 10, 0)
    assert d.size == 0
    with pytest.raises(ValueError):
        o.draw_indices(4, 0, 3, 4)


def test_gather_intersection_invariant():
    A = synth.plain_lowrank(50, 40, 3).astype(np.float32)
    rows, cols = np.array([1, 7, 30]), np.array([0, 5, 39, 22])
    pins.pin_gather_intersection(o.gather_dense, A, rows, cols)
    X, Y, sig = synth.rbf_mixture(31, 40, d=4, components=3, sigma_pairs=50)
    C, Rt, W = o.gather_rbf(X, Y, sig, rows, cols)
    assert np.array_equal(W, C[rows, :]) and np.array_equal(W, Rt[cols, :].T)


def test_rbf_entry_closed_forms():
    pins.pin_rbf_closed_forms(o.rbf_entries)


def test_rbf_block_and_gather_match_entries():
    pins.pin_rbf_block_and_gather(o.rbf_block, o.gather_rbf, o.rbf_entries)


def test_upsilon_weights_closed_form():
    pins.pin_upsilon_weights(o.upsilon_weights)


def test_encoding_error_closed_form():
    pins.pin_encoding_error_closed_form(o.encoding_error)


def test_sampled_error_closed_form():
    pins.pin_sampled_error_closed_form(o.rel_fro_error_sampled, o.DenseSource)


def test_pinv_exact_recovery_rank_k():
    pins.pin_pinv_exact_recovery(o.gather_dense, o.sketching)
    pins.pin_pinv_exact_recovery(o.gather_dense, o.sketching, m=80, n=33, r=8, k=8, seed=5)


def test_pinv_equals_pseudoskeleton():
    pins.pin_pinv_equals_pseudoskeleton(o.gather_dense, o.sketching)


def test_stabilized_rank1_closed_form():
    pins.pin_stabilized_rank1_closed_form(o.gather_dense, o.sketching)


def test_stabilized_rank2_closed_form():
    pins.pin_stabilized_rank2_hadamard(o.gather_dense, o.sketching)


def test_unit_columns_truncation_and_svd():
    pins.pin_unit_columns_and_truncation(o.gather_dense, o.sketching)


def test_embed_closed_form_and_pseudoskeleton():
    pins.pin_embed(o.embed, o.sketching, o.gather_dense)


def test_kmeans_bruteforce_optimum():
    pins.pin_kmeans_bruteforce_optimum(o.weighted_kmeans)


def test_kmeans_steps_exhaustive():
    pins.pin_kmeans_steps_exhaustive(o.weighted_kmeans)
    pins.pin_kmeans_steps_exhaustive(o.weighted_kmeans, p=0.0, seed=4)


def test_kmeans_ties_and_empty_clusters():
    pins.pin_kmeans_ties_and_empty(o.weighted_kmeans)


def test_kmeans_matches_sklearn():
    pins.pin_kmeans_matches_sklearn(o.weighted_kmeans)


def test_snap_bruteforce():
    pins.pin_snap_bruteforce(o.snap)


def test_snap_midpoint_tie():
    pins.pin_snap_midpoint_tie(o.snap)


def test_threshold_bruteforce_and_known_scales():
    pins.pin_threshold_bruteforce(o.hard_threshold)
    pins.pin_threshold_known_scales(o.hard_threshold)


def test_error_closed_form():
    pins.pin_error_closed_form(o.rel_fro_error_dense)


def test_philox_published_known_answers():
    """Known-answer vectors published with Philox (Salmon et al., SC'11)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.txt")
    n = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        lhs, rhs = line.split(":")
        w = [int(x, 16) for x in lhs.split()]
        want = tuple(int(x, 16) for x in rhs.split())
        assert o.philox4x64_10(w[:4], w[4:6]) == want
        n += 1
    assert n == 3


def test_plain_fp64_regression_fixture():
    """The oracle still produces the committed output on the plain FP64 workload."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "plain_fp64_2000x1500_k20.json")
    gold = json.load(open(path))
    A = synth.plain_lowrank()
    for mode, g in gold.items():
        r = o.cabs(o.DenseSource(A), k1=20, iters=5, seed=1607, mode=mode)
        assert r.pilot_rows.tolist() == g["pilot_rows"] and r.pilot_cols.tolist() == g["pilot_cols"]
        assert r.rows.tolist() == g["rows"] and r.cols.tolist() == g["cols"]
        assert abs(o.rel_fro_error_dense(A, r.final.U, r.final.S, r.final.V) - g["final_err"]) <= 1e-9 * g["final_err"]


def test_orthogonalize():
    pins.pin_orthogonalize(o.orthogonalize)


def test_pinv_trunc():
    pins.pin_pinv_trunc(o.pinv_trunc)


def test_br_cur():
    pins.pin_br_cur(o.br_cur, o.DenseSource)


def test_sketch_cur_draws():
    """Sketch-CUR draws k_b base and 3 k_b target indices per side, distinct,
    sorted, inside the matrix; an exactly rank-3 matrix is recovered."""
    from workloads import synth
    A = synth.exact_lowrank_int(300, 200, 3, seed=4)
    r = o.sketch_cur(o.DenseSource(A), 5, seed=11)
    for idx, k, N in ((r.rows_b, 5, 300), (r.cols_b, 5, 200), (r.rows_t, 15, 300), (r.cols_t, 15, 200)):
        assert len(idx) == k and len(set(idx.tolist())) == k and np.all(np.diff(idx) > 0)
        assert idx.min() >= 0 and idx.max() < N
    assert not np.array_equal(r.rows_b, r.rows_t[:5])
    assert np.allclose(r.C @ r.U @ r.Rt.T, A, atol=1e-9 * np.abs(A).max())


def test_leverage_scores():
    pins.pin_leverage_scores(o.leverage_scores, o.orthogonalize)


def test_weighted_sample():
    pins.pin_weighted_sample(o.weighted_sample)


def test_philox_uniform_matches_numpy():
    assert np.array_equal(o.philox_uniform(11, 6, 9), pins.philox_uniform_for_pin(11, 6, 9))


def test_leverage_follow_up_sketch():
    """Section 5 variant (e) end to end on an exactly rank-3 matrix whose
    rows 0..99 are zero: those rows have leverage 0 and are never drawn, the
    indices are distinct and sorted, and the follow-up sketch recovers A."""
    from workloads import synth
    A = synth.exact_lowrank_int(400, 300, 3, seed=2)
    A[:100] = 0.0
    r = o.cabs(o.DenseSource(A), 12, 6, seed=5, follow="leverage")
    assert r.rows.min() >= 100 and len(set(r.rows.tolist())) == 6 and np.all(np.diff(r.rows) > 0)
    assert len(set(r.cols.tolist())) == 6 and np.all(np.diff(r.cols) > 0)
    F = r.final
    assert np.allclose((F.U * F.S) @ F.V.T, A, atol=1e-8 * np.abs(A).max())


def test_csr_source_matches_dense():
    """The sparse source's gathers and entries (scipy's sparse slicing) equal
    the dense source's on the densified matrix, bit for bit; rows with no
    stored entries gather as zeros."""
    from workloads import synth
    ip, ix, v = synth.sparse_lowrank(300, 200, 0.03, rank=4, seed=3)
    src = o.CSRSource(ip, ix, v, 200)
    A = src.dense()
    assert A.shape == (300, 200) and np.count_nonzero(A) == len(v)
    dense = o.DenseSource(A)
    g = np.random.default_rng(2)
    rows = np.sort(g.choice(300, 17, replace=False))
    cols = np.sort(g.choice(200, 13, replace=False))
    for a, b in zip(src.gather(rows, cols), dense.gather(rows, cols)):
        assert np.array_equal(a, b)
    ii, jj = g.integers(0, 300, 500), g.integers(0, 200, 500)
    assert np.array_equal(src.entries(ii, jj), dense.entries(ii, jj))
    # sketches of the two sources agree exactly (same arithmetic downstream)
    r1 = o.cabs(src, 12, 8, seed=5)
    r2 = o.cabs(dense, 12, 8, seed=5)
    assert np.array_equal(r1.rows, r2.rows) and np.array_equal(r1.cols, r2.cols)
    assert np.array_equal(r1.final.U, r2.final.U)


def test_sparse_error_identity():
    """|A - L|^2 = |A|^2 - 2 <A, L>_stored + sum_pq S_p S_q (U^T U)_pq (V^T V)_pq,
    the linear-cost form of the exact error for a sparse A, equals the dense
    definition."""
    from workloads import synth
    ip, ix, v = synth.sparse_lowrank(150, 120, 0.05, rank=3, seed=8)
    src = o.CSRSource(ip, ix, v, 120)
    A = src.dense()
    g = np.random.default_rng(4)
    U, V, S = g.standard_normal((150, 6)), g.standard_normal((120, 6)), np.abs(g.standard_normal(6))
    L = (U * S) @ V.T
    rows = np.repeat(np.arange(150), np.diff(ip))
    cross = np.sum(v.astype(np.float64) * L[rows, ix])
    l2 = np.sum(np.outer(S, S) * (U.T @ U) * (V.T @ V))
    num = np.sum(v.astype(np.float64) ** 2) - 2 * cross + l2
    want = o.rel_fro_error_dense(A, U, S, V)
    assert abs(np.sqrt(num / np.sum(A ** 2)) - want) < 1e-12 * want


def test_philox_uniform_definition():
    pins.pin_philox_uniform(o.philox_uniform)


def test_eval_samples_definition():
    pins.pin_eval_samples(o.eval_samples)


def test_sq_dists_closed_form():
    pins.pin_sq_dists(o.sq_dists_to)


def test_csr_gather_against_explicit_dense():
    pins.pin_csr_gather(o.CSRSource, o.DenseSource)
