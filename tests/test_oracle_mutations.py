"""Plants plausible mistakes in copies of oracle functions and checks that the
pins reject every one of them (a dropped term, a wrong sign or index, a
transposed operand). Runs on the CPU only; the oracle itself is not modified."""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import cabs_ref as o
from tests import oracle_pins as pins


def mutate(fn, old, new):
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, (fn.__name__, old)
    ns = dict(o.__dict__)
    exec(compile(src.replace(old, new), f"<mutant {fn.__name__}>", "exec"), ns)
    return ns[fn.__name__]


def rejects(check):
    try:
        check()
    except (AssertionError, IndexError, ValueError, ZeroDivisionError, FloatingPointError):
        return True
    return False


SKETCH_MUTANTS = [
    ("a = C @ Vw[:, :r]", "a = C @ Uw[:, :r]"),                         # transposed factor
    ("b = Rt @ Uw[:, :r]", "b = Rt @ Vw[:, :r]"),
    ("S[i] = Nc[i] * Nr[i] / sig[i]", "S[i] = Nc[i] * Nr[i] * sig[i]"),  # wrong exponent
    ("S[i] = Nc[i] * Nr[i] / sig[i]", "S[i] = Nc[i] / sig[i]"),          # dropped term
    ("S[i] = sig[i] * math.sqrt(m * n / (k_r * k_c))", "S[i] = sig[i]"),  # dropped scale
    ("S[i] = sig[i] * math.sqrt(m * n / (k_r * k_c))", "S[i] = sig[i] * math.sqrt(m * n) / (k_r * k_c)"),
    ("V[:, i] = b[:, i] / Nr[i]", "V[:, i] = b[:, i]"),                  # dropped normalisation
    ("r = int(np.count_nonzero(sig > tol))", "r = int(np.count_nonzero(sig >= 0))"),  # no truncation
]


@pytest.mark.parametrize("old,new", SKETCH_MUTANTS)
def test_sketching_mutants_rejected(old, new):
    bad = mutate(o.sketching, old, new)
    checks = [lambda: pins.pin_pinv_exact_recovery(o.gather_dense, bad),
              lambda: pins.pin_pinv_equals_pseudoskeleton(o.gather_dense, bad),
              lambda: pins.pin_stabilized_rank1_closed_form(o.gather_dense, bad),
              lambda: pins.pin_stabilized_rank2_hadamard(o.gather_dense, bad),
              lambda: pins.pin_unit_columns_and_truncation(o.gather_dense, bad)]
    assert any(rejects(c) for c in checks)


@pytest.mark.parametrize("old,new", [
    ("Rt = np.array(A[rows, :].T, dtype=np.float64)", "Rt = np.array(A[:, rows], dtype=np.float64)"),
    ("W = np.array(A[np.ix_(rows, cols)], dtype=np.float64)", "W = np.array(A[np.ix_(cols, rows)].T, dtype=np.float64)"),
])
def test_gather_mutants_rejected(old, new):
    bad = mutate(o.gather_dense, old, new)
    A = np.arange(60.0).reshape(6, 10)
    assert rejects(lambda: pins.pin_gather_intersection(bad, A, np.array([1, 4]), np.array([0, 3, 9])))


@pytest.mark.parametrize("old,new", [
    ("for _ in range(10):", "for _ in range(9):"),
    ("k0 = (k0 + _W0) & MASK64", "k0 = (k0 + _W1) & MASK64"),
    ("c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK64, (p0 >> 64) ^ c3 ^ k1, p0 & MASK64)",
     "c0, c1, c2, c3 = ((p0 >> 64) ^ c1 ^ k0, p1 & MASK64, (p1 >> 64) ^ c3 ^ k1, p0 & MASK64)"),
])
def test_philox_mutants_rejected(old, new):
    bad = mutate(o.philox4x64_10, old, new)
    assert rejects(lambda: pins.pin_philox_matches_numpy(bad))


@pytest.mark.parametrize("old,new", [
    ("j = i + mulhi64(r, N - i)", "j = i + mulhi64(r, N)"),
    ("j = i + mulhi64(r, N - i)", "j = mulhi64(r, N - i)"),
    ("moved[j] = vi", "moved[j] = vj"),
])
def test_draw_mutants_rejected(old, new):
    bad = mutate(o.draw_indices, old, new)
    assert rejects(lambda: pins.pin_draw_is_partial_fisher_yates(bad, o.philox4x64_10)) or \
        rejects(lambda: pins.pin_draw_uniform(bad, trials=500))


@pytest.mark.parametrize("old,new", [
    ("Znew[j] = (w[mem, None] * X[mem]).sum(axis=0) / wsum", "Znew[j] = X[mem].mean(axis=0)"),  # weights dropped
    ("s = np.argmin(D, axis=1)", "s = D.shape[1] - 1 - np.argmin(D[:, ::-1], axis=1)"),         # ties to highest
    ("Znew = Z.copy()", "Znew = np.zeros_like(Z)"),                                             # empty -> origin
    ("res.energy.append(float((w * best).sum()))", "res.energy.append(float(best.sum()))"),      # unweighted energy
])
def test_kmeans_mutants_rejected(old, new):
    bad = mutate(o.weighted_kmeans, old, new)
    checks = [lambda: pins.pin_kmeans_steps_exhaustive(bad),
              lambda: pins.pin_kmeans_ties_and_empty(bad),
              lambda: pins.pin_kmeans_bruteforce_optimum(bad, trials=3)]
    assert any(rejects(c) for c in checks)


SNAP_PICK = "l = int(np.flatnonzero(d <= dstar + tie_rtol * (dstar + float((z * z).sum())))[0])"


@pytest.mark.parametrize("old,new", [
    ("d[taken] = np.inf", "pass"),
    ("taken[l] = True", "taken[l] = False"),
    (SNAP_PICK, "l = int(np.argmin(d))"),                                          # rounding decides ties
    (SNAP_PICK, SNAP_PICK.replace("[0])", "[-1])")),                                # ties to the highest row
    (SNAP_PICK, SNAP_PICK.replace("tie_rtol *", "1e3 * tie_rtol *")),              # window wider than rounding
    (SNAP_PICK, SNAP_PICK.replace("(dstar + float((z * z).sum()))", "dstar")),     # no |z|^2 scale
])
def test_snap_mutants_rejected(old, new):
    bad = mutate(o.snap, old, new)
    assert rejects(lambda: pins.pin_snap_bruteforce(bad)) or rejects(lambda: pins.pin_snap_midpoint_tie(bad))


@pytest.mark.parametrize("old,new", [
    ("return U * np.sqrt(S)[None, :]", "return U * S[None, :]"),            # U S
    ("return U * np.sqrt(S)[None, :]", "return U * (S ** 2)[None, :]"),     # U S^2
    ("return U * np.sqrt(S)[None, :]", "return U * np.sqrt(S[::-1])[None, :]"),  # scales on the wrong columns
])
def test_embed_mutants_rejected(old, new):
    bad = mutate(o.embed, old, new)
    assert rejects(lambda: pins.pin_embed(bad, o.sketching, o.gather_dense))


def test_error_mutant_rejected():
    bad = mutate(o.rel_fro_error_dense, "return math.sqrt(num / den) if den > 0 else 0.0",
                 "return num / den if den > 0 else 0.0")
    assert rejects(lambda: pins.pin_error_closed_form(bad))


THRESHOLD_MUTANTS = [
    ("order = np.lexsort((np.arange(M), -sq))", "order = np.lexsort((np.arange(M), sq))"),      # smallest
    ("order = np.lexsort((np.arange(M), -sq))", "order = np.lexsort((-np.arange(M), -sq))"),    # ties high
    ("sq = sq + X[:, q] * X[:, q]", "sq = sq + X[:, q]"),                                       # not a norm
    ("return np.sort(order[:k2]).astype(np.int64)", "return order[:k2].astype(np.int64)"),      # unsorted
]


@pytest.mark.parametrize("old,new", THRESHOLD_MUTANTS)
def test_threshold_mutants_rejected(old, new):
    bad = mutate(o.hard_threshold, old, new)
    assert rejects(lambda: (pins.pin_threshold_bruteforce(bad), pins.pin_threshold_known_scales(bad)))


ORTH_MUTANTS = [
    ("B = (s0[:, None] * V0t) @ (S[:, None] * V.T)", "B = (s0[:, None] * V0t) @ (S[:, None] * V).T"),  # wrong shape use
    ("B = (s0[:, None] * V0t) @ (S[:, None] * V.T)", "B = V0t @ (S[:, None] * V.T)"),                   # dropped Sigma_0
    ("B = (s0[:, None] * V0t) @ (S[:, None] * V.T)", "B = (s0[:, None] * V0t.T) @ (S[:, None] * V.T)"),  # transposed V_0
    ("return U0 @ U1[:, keep], s1[keep], V1t.T[:, keep]", "return U0[:, keep], s1[keep], V1t.T[:, keep]"),  # dropped U_1
    ("return U0 @ U1[:, keep], s1[keep], V1t.T[:, keep]", "return U0 @ U1[:, keep], s1[keep], V1t[:, keep]"),
]


@pytest.mark.parametrize("old,new", ORTH_MUTANTS)
def test_orthogonalize_mutants_rejected(old, new):
    bad = mutate(o.orthogonalize, old, new)
    assert rejects(lambda: pins.pin_orthogonalize(bad))


CUR_MUTANTS = [
    ("Cbar = C[rows_t, :]", "Cbar = C[rows_t[::-1], :]"),                      # rows out of order
    ("Rbar = Rt[cols_t, :].T", "Rbar = Rt[cols_t, :].T[:, ::-1]"),
    ("Ustar = pinv_trunc(Cbar, trunc_rtol) @ M @ pinv_trunc(Rbar, trunc_rtol)",
     "Ustar = pinv_trunc(Cbar, trunc_rtol) @ M.T @ pinv_trunc(Rbar, trunc_rtol)"),  # transposed target
    ("Ustar = pinv_trunc(Cbar, trunc_rtol) @ M @ pinv_trunc(Rbar, trunc_rtol)",
     "Ustar = Cbar.T @ M @ pinv_trunc(Rbar, trunc_rtol)"),                      # transpose for pinv
]

PINV_MUTANTS = [
    ("keep = sb > max(trunc_rtol, max(B.shape) * EPS64) * sb[0]",
     "keep = sb > max(trunc_rtol, min(B.shape) * EPS64) * sb[0]"),
    ("keep = sb > max(trunc_rtol, max(B.shape) * EPS64) * sb[0]",
     "keep = sb > max(trunc_rtol, math.sqrt(max(B.shape) * EPS64)) * sb[0]"),
    ("return (Vbt[keep].T / sb[keep]) @ Ub[:, keep].T", "return (Vbt[keep].T * sb[keep]) @ Ub[:, keep].T"),
    ("return (Vbt[keep].T / sb[keep]) @ Ub[:, keep].T", "return (Vbt[keep] / sb[keep][:, None]).T @ Ub[:, keep].T[::-1]"),
]


@pytest.mark.parametrize("old,new", CUR_MUTANTS)
def test_br_cur_mutants_rejected(old, new):
    bad = mutate(o.br_cur, old, new)
    assert rejects(lambda: pins.pin_br_cur(bad, o.DenseSource))


@pytest.mark.parametrize("old,new", PINV_MUTANTS)
def test_pinv_mutants_rejected(old, new):
    bad = mutate(o.pinv_trunc, old, new)
    assert rejects(lambda: pins.pin_pinv_trunc(bad))


WS_MUTANTS = [
    ("keys = w / -np.log(u)", "keys = w * -np.log(u)"),                  # inverted key map
    ("keys = w / -np.log(u)", "keys = w / -np.log(1 - u)"),              # other uniform
    ("order = np.lexsort((np.arange(N), -keys))", "order = np.lexsort((np.arange(N), keys))"),  # smallest keys
]


@pytest.mark.parametrize("old,new", WS_MUTANTS)
def test_weighted_sample_mutants_rejected(old, new):
    bad = mutate(o.weighted_sample, old, new)
    assert rejects(lambda: pins.pin_weighted_sample(bad))


LEV_MUTANTS = [
    ("return (X * X).sum(axis=1)", "return np.abs(X).sum(axis=1)"),
    ("return (X * X).sum(axis=1)", "return (X * X).sum(axis=0)"),
]


@pytest.mark.parametrize("old,new", LEV_MUTANTS)
def test_leverage_mutants_rejected(old, new):
    bad = mutate(o.leverage_scores, old, new)
    assert rejects(lambda: pins.pin_leverage_scores(bad, o.orthogonalize))


RBF_ENTRY_MUTANTS = [
    ("return np.exp(-d2 / (2.0 * s * s))", "return np.exp(-d2 / (s * s))"),       # sigma^2 for 2 sigma^2
    ("return np.exp(-d2 / (2.0 * s * s))", "return np.exp(-d2 / (2.0 * s))"),     # sigma for sigma^2
    ("d2 = ((x - y) ** 2).sum(axis=-1)", "d2 = np.abs(x - y).sum(axis=-1)"),      # L1 distance
]


@pytest.mark.parametrize("old,new", RBF_ENTRY_MUTANTS)
def test_rbf_entry_mutants_rejected(old, new):
    bad = mutate(o.rbf_entries, old, new)
    assert rejects(lambda: pins.pin_rbf_closed_forms(bad))


RBF_BLOCK = "out[:, t] = np.exp(-((x - y[t]) ** 2).sum(axis=1) / (2.0 * s * s))"
RBF_GATHER_MUTANTS = [
    ("C = rbf_block(X, Y, sigma, np.arange(m), cols)", "C = rbf_block(X, Y, sigma, np.arange(m), rows)"),
    ("Rt = rbf_block(X, Y, sigma, rows, np.arange(n)).T.copy()",
     "Rt = rbf_block(X, Y, sigma, cols, np.arange(n)).T.copy()"),
    ("W = rbf_block(X, Y, sigma, rows, cols)", "W = rbf_block(X, Y, sigma, rows, cols[::-1])"),
]


@pytest.mark.parametrize("old,new", [(RBF_BLOCK, RBF_BLOCK.replace("2.0 * s * s", "s * s")),
                                     (RBF_BLOCK, RBF_BLOCK.replace("y[t]", "y[0]"))])
def test_rbf_block_mutants_rejected(old, new):
    bad = mutate(o.rbf_block, old, new)
    assert rejects(lambda: pins.pin_rbf_block_and_gather(bad, o.gather_rbf, o.rbf_entries))


@pytest.mark.parametrize("old,new", RBF_GATHER_MUTANTS)
def test_rbf_gather_mutants_rejected(old, new):
    bad = mutate(o.gather_rbf, old, new)
    assert rejects(lambda: pins.pin_rbf_block_and_gather(o.rbf_block, bad, o.rbf_entries))


@pytest.mark.parametrize("old,new", [
    ("nrm = np.sqrt((X * X).sum(axis=1))", "nrm = (X * X).sum(axis=1)"),          # squared norm
    ("nrm = np.sqrt((X * X).sum(axis=1))", "nrm = np.sqrt((X * X).sum(axis=0))"),  # column norms
    ("return nrm ** p", "return nrm ** (p / 2)"),
])
def test_upsilon_mutants_rejected(old, new):
    bad = mutate(o.upsilon_weights, old, new)
    assert rejects(lambda: pins.pin_upsilon_weights(bad))


ENC_ERR = "err = float((w * D[np.arange(X.shape[0]), s]).sum())"


@pytest.mark.parametrize("old,new", [
    (ENC_ERR, ENC_ERR.replace("w * ", "")),                                       # weights dropped
    ("s = np.argmin(D, axis=1)", "s = np.argmax(D, axis=1)"),                     # farthest representative
    ("T = int(np.bincount(s, minlength=Z.shape[0]).max())", "T = int(np.bincount(s, minlength=Z.shape[0]).min())"),
])
def test_encoding_error_mutants_rejected(old, new):
    bad = mutate(o.encoding_error, old, new)
    assert rejects(lambda: pins.pin_encoding_error_closed_form(bad))


SAMPLED_US = "US = np.asarray(U, dtype=np.float64) * np.asarray(S, dtype=np.float64)[None, :]"
SAMPLED_AHAT = "ahat = (US[ii] * np.asarray(V, dtype=np.float64)[jj]).sum(axis=1)"


@pytest.mark.parametrize("old,new", [
    ("return math.sqrt(num / den) if den > 0 else 0.0", "return num / den if den > 0 else 0.0"),  # no square root
    (SAMPLED_US, "US = np.asarray(U, dtype=np.float64)"),                                          # S dropped
    (SAMPLED_AHAT, SAMPLED_AHAT.replace("[jj]", "[ii]")),                                          # wrong index
])
def test_sampled_error_mutants_rejected(old, new):
    bad = mutate(o.rel_fro_error_sampled, old, new)
    assert rejects(lambda: pins.pin_sampled_error_closed_form(bad, o.DenseSource))


DRIVER_MUTANTS = [
    ("Cb, Rtb, Wb = source.gather(rows, cols)", "Cb, Rtb, Wb = source.gather(Ir, Ic)"),            # no follow-up gather
    ("rows_o, rows = snap(P, km_r.Z)", "rows_o, rows = snap(P, km_r.centres[0])"),                 # k-means skipped
    ("P = embed(pilot.U, pilot.S)", "P = pilot.U"),                                                # no embedding
    ("km_c = weighted_kmeans(Q, Ic_drawn[:k2], iters, upsilon_pow)",
     "km_c = weighted_kmeans(Q, Ic[:k2], iters, upsilon_pow)"),                                   # sorted, not drawn
]


@pytest.mark.parametrize("old,new", DRIVER_MUTANTS)
def test_driver_mutants_rejected(old, new):
    bad = mutate(o.cabs, old, new)
    checks = [lambda: pins.pin_driver_wiring(bad, o.DenseSource, o.sketching, o.embed, o.weighted_kmeans, o.snap),
              lambda: pins.pin_follow_up_improves_encoding(bad, o.DenseSource, trials=4)]
    assert any(rejects(c) for c in checks)


PU = "return ((r0 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53"


@pytest.mark.parametrize("old,new", [
    (PU, PU.replace(" + 0.5", "")),                                                    # u = 0 possible
    (PU, PU.replace("np.uint64(11)", "np.uint64(12)")),                                # wrong shift
    ("r0 = philox4x64_10_vec(c0, z, z, z, seed, tag)[0]", "r0 = philox4x64_10_vec(c0, z, z, z, seed, tag)[1]"),
])
def test_philox_uniform_mutants_rejected(old, new):
    bad = mutate(o.philox_uniform, old, new)
    assert rejects(lambda: pins.pin_philox_uniform(bad))


ES_RET = "return mulhi64_vec(w0, m).astype(np.int64), mulhi64_vec(w1, n).astype(np.int64)"


@pytest.mark.parametrize("old,new", [
    (ES_RET, "return mulhi64_vec(w1, m).astype(np.int64), mulhi64_vec(w0, n).astype(np.int64)"),  # words swapped
    (ES_RET, "return (w0 % np.uint64(m)).astype(np.int64), (w1 % np.uint64(n)).astype(np.int64)"),  # modulo map
    ("w0, w1, _, _ = philox4x64_10_vec(t, z, z, z, seed, TAG_EVAL)",
     "w0, w1, _, _ = philox4x64_10_vec(t, z, z, z, seed, TAG_ROWS)"),                               # wrong key
])
def test_eval_samples_mutants_rejected(old, new):
    bad = mutate(o.eval_samples, old, new)
    assert rejects(lambda: pins.pin_eval_samples(bad))


@pytest.mark.parametrize("old,new", [
    ("d = X - z[None, :]", "d = X + z[None, :]"),
    ("return (d * d).sum(axis=1)", "return np.abs(d).sum(axis=1)"),
])
def test_sq_dists_mutants_rejected(old, new):
    bad = mutate(o.sq_dists_to, old, new)
    assert rejects(lambda: pins.pin_sq_dists(bad))


@pytest.mark.parametrize("old,new", [
    ("C = np.asarray(self.A[:, cols].toarray(), dtype=np.float64)",
     "C = np.asarray(self.A[:, rows].toarray(), dtype=np.float64)"),                       # wrong index set
    ("Rt = np.asarray(self.A[rows, :].toarray().T, dtype=np.float64)",
     "Rt = np.asarray(self.A[rows, :].toarray(), dtype=np.float64)"),                      # not transposed
    ("W = np.asarray(self.A[rows, :][:, cols].toarray(), dtype=np.float64)",
     "W = np.asarray(self.A[cols, :][:, rows].toarray().T, dtype=np.float64)"),            # transposed intersection
])
def test_csr_gather_mutants_rejected(old, new):
    bad = mutate(o.CSRSource.gather, old, new)
    Bad = type("Bad", (o.CSRSource,), {"gather": bad})
    assert rejects(lambda: pins.pin_csr_gather(Bad, o.DenseSource))
