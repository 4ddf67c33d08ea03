"""Algorithm 2 end to end on the oracle: exact cases and statistical properties (no GPU)."""
import math

import numpy as np

from oracle import cabs_ref as o
from tests import oracle_pins as pins
from workloads import synth


def test_cabs_exact_rank_recovery():
    """An exactly rank-r matrix with k >= r is recovered by both rounds (pinv core)."""
    A = synth.exact_lowrank_int(120, 90, 6, seed=21)
    res = o.cabs(o.DenseSource(A), k1=10, iters=3, seed=5)
    assert res.pilot.rank == 6 and res.final.rank == 6
    assert o.rel_fro_error_dense(A, res.pilot.U, res.pilot.S, res.pilot.V) < 1e-10
    assert o.rel_fro_error_dense(A, res.final.U, res.final.S, res.final.V) < 1e-10
    assert len(set(res.rows.tolist())) == 10 and np.all(np.diff(res.rows) > 0)


def test_cabs_threshold_follow_up():
    """The hard-threshold variant (Section 5): the follow-up rows are the k2
    largest-norm rows of P (and columns of Q), and an exactly rank-r matrix is
    still recovered exactly by the final round (any rows and columns with
    rank(W_bar) = r do that)."""
    A = synth.exact_lowrank_int(120, 90, 6, seed=21)
    res = o.cabs(o.DenseSource(A), k1=10, iters=3, seed=5, follow="threshold")
    nP = (res.P ** 2).sum(1)
    assert set(res.rows.tolist()) == set(np.argsort(-nP, kind="stable")[:10].tolist())
    assert res.km_rows is None and len(set(res.cols.tolist())) == 10
    assert res.final.rank == 6
    assert o.rel_fro_error_dense(A, res.final.U, res.final.S, res.final.V) < 1e-10


def test_cabs_init_uses_pilot_rows_in_draw_order():
    A = synth.plain_lowrank(200, 150, 5)
    res = o.cabs(o.DenseSource(A), k1=8, k2=5, iters=2, seed=3)
    assert np.array_equal(res.km_rows.centres[0], res.P[res.pilot_rows_drawn[:5]])
    assert np.array_equal(res.km_cols.centres[0], res.Q[res.pilot_cols_drawn[:5]])


def test_follow_up_encoding_error_drops():
    """e_f < e_p (the premise of Theorem 2) on at least 95% of seeds."""
    pins.pin_follow_up_improves_encoding(o.cabs, o.DenseSource)


def test_driver_composes_the_steps_in_order():
    pins.pin_driver_wiring(o.cabs, o.DenseSource, o.sketching, o.embed, o.weighted_kmeans, o.snap)


def test_sampled_error_within_three_standard_errors():
    X, Y, sig = synth.rbf_mixture(400, 300, d=4, components=5, sigma_pairs=200)
    src = o.RBFSource(X, Y, sig)
    res = o.cabs(src, k1=12, iters=3, seed=2)
    U, S, V = res.final.U, res.final.S, res.final.V
    A = o.rbf_block(X, Y, sig, np.arange(400), np.arange(300))
    exact = o.rel_fro_error_dense(A, U, S, V)
    ii, jj = o.eval_samples(7, 400, 300, 20000)
    a = src.entries(ii, jj)
    ah = ((U * S)[ii] * V[jj]).sum(1)
    est = o.rel_fro_error_sampled(src, U, S, V, 7, 20000)
    # delta method on sqrt(mean(num) / mean(den))
    num, den = (a - ah) ** 2, a * a
    cov = np.cov(np.vstack([num, den])) / len(a)
    g = np.array([1 / den.mean(), -num.mean() / den.mean() ** 2]) / (2 * est)
    se = math.sqrt(g @ cov @ g)
    assert abs(est - exact) <= 3 * se + 1e-12


def test_eval_samples_uniform():
    from scipy.stats import chisquare
    ii, jj = o.eval_samples(3, 17, 11, 17000)
    assert ii.min() >= 0 and ii.max() < 17 and jj.min() >= 0 and jj.max() < 11
    assert chisquare(np.bincount(ii, minlength=17)).pvalue > 1e-4
    assert chisquare(np.bincount(jj, minlength=11)).pvalue > 1e-4
