"""Tensor-core (tcgen05) paths against the FP64 oracle: the fused residual,
the k-means assignment, and whole sketches in BF16 / TF32 mode.

Tolerances follow the operand rounding: BF16 operands carry 2^-8 relative
error, TF32 (possibly truncated) 2^-10; the residual's relative error on a sketch with error >= 0.05
moves by far less than 1e-3 of itself; assignments differ from FP64 only on
rows the re-check cannot separate (counted, must be rare)."""
import numpy as np
import pytest

from oracle import cabs_ref as o
from workloads import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1607_07395_gb300 import cabs
    return cabs


@pytest.fixture(scope="module")
def ctx(C):
    assert torch.cuda.is_available()
    return C.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def fake_result(C, U, S, V, p):
    sk = C.alloc_result(p)
    sk.U.copy_(dev(U.astype(np.float32)))
    sk.S.copy_(dev(S.astype(np.float64)))
    sk.V.copy_(dev(V.astype(np.float32)))
    return sk


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("m,n,lda,k", [(1000, 700, 700, 20), (4096, 2048, 2048, 256), (777, 1333, 1400, 100),
                                       (130, 300, 304, 65), (5000, 257, 257, 128)])
def test_tc_residual_matches_exact(ctx, C, prec, m, n, lda, k):
    if prec == "tf32" and k > 256:
        pytest.skip()
    g = np.random.default_rng(m + n + k)
    r = min(k, 40)
    L = g.standard_normal((m, r)) @ g.standard_normal((r, n)) / np.sqrt(r)
    full = np.zeros((m, lda), dtype=np.float32)
    full[:, :n] = (L + 0.3 * g.standard_normal((m, n))).astype(np.float32)
    A = full[:, :n].astype(np.float64)
    U = g.standard_normal((m, k))
    V = g.standard_normal((n, k))
    U /= np.linalg.norm(U, axis=0)
    V /= np.linalg.norm(V, axis=0)
    S = np.abs(g.standard_normal(k)) * np.sqrt(m * n) / k
    p = C.make_params(m, n, k, prec=prec)
    sk = fake_result(C, U, S, V, p)
    Ad = dev(full)[:, :n]
    got = C.cabs_error(ctx, C.dense_source(Ad), p, sk)
    want = o.rel_fro_error_dense(A, U.astype(np.float32).astype(np.float64), S,
                                 V.astype(np.float32).astype(np.float64))
    assert abs(got / want - 1) <= 1e-3, (got, want)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,d,k2", [(2000, 20, 20), (9000, 64, 64), (4099, 128, 100), (70000, 64, 256),
                                    (9001, 256, 256), (5000, 200, 200), (3001, 160, 129), (2000, 256, 100)])
def test_tc_assign_matches_oracle(ctx, C, prec, M, d, k2):
    g = np.random.default_rng(M + d)
    centers = 3.0 * g.standard_normal((50, d))
    X = centers[g.integers(0, 50, M)] + g.standard_normal((M, d))
    init = g.choice(M, k2, replace=False)
    ref = o.weighted_kmeans(X.astype(np.float32).astype(np.float64), init, 3, 0.0)
    out = C.cabs_kmeans(ctx, dev(X.astype(np.float32)), dev(init.astype(np.int32)), k2, 3, prec=prec)
    lab = out["labels"].cpu().numpy()
    # iteration 0 sees the same centres on both sides: labels agree except unresolved near-ties
    mism = (lab[0] != ref.labels[0]).mean()
    assert mism <= 1e-3, mism
    e = out["energy"].cpu().numpy()
    assert np.all(np.abs(e / np.array(ref.energy) - 1) <= 1e-3), (e, ref.energy)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_sketch_reduced_precision_excess_small(ctx, C, prec):
    A, _, _, _ = synth.decaying_lowrank_host(4096, 2048, rank=256, decay=30, noise_std=1e-4, seed=1607)
    k = 64 if prec == "tf32" else 128
    ref = o.cabs(o.DenseSource(A), k, iters=5, seed=1607, mode="stabilized")
    e_ref = o.rel_fro_error_dense(A, ref.final.U, ref.final.S, ref.final.V)
    p = C.make_params(4096, 2048, k, iters=5, seed=1607, prec=prec, core="stabilized")
    Ad = dev(A)
    sk = C.cabs_sketch(ctx, C.dense_source(Ad), p)
    e = C.cabs_error(ctx, C.dense_source(Ad), p, sk)
    assert sk.pilot_rows.cpu().numpy().tolist() == ref.pilot_rows.tolist()
    assert e / e_ref - 1 <= 1e-3, (e, e_ref)
    d = sk.diag()
    assert d.status == 0


# ------------------------------------------- a6: snap in reduced precision

def to_np(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("M,d,k2", [(5000, 64, 64), (777, 20, 7), (3000, 128, 200), (2500, 256, 256),
                                    (70000, 100, 150), (5, 3, 3)])
def test_tc_snap_matches_oracle(ctx, C, prec, M, d, k2):
    """In the reduced-precision modes the snap still decides by direct
    distances, so it gives the oracle's greedy picks (Section 3.2) on data
    whose nearest rows are separated."""
    if prec == "tf32" and d > 128:
        pytest.skip("TF32 operands are limited to width 128")
    g = np.random.default_rng(M + 7 * d + k2)
    X = g.standard_normal((M, d)).astype(np.float32)
    Z = (X[g.choice(M, k2, replace=False)] + 0.3 * g.standard_normal((k2, d))).astype(np.float32)
    order, srt = C.cabs_snap(ctx, dev(X), dev(Z), prec=prec)
    want_o, want_s = o.snap(X.astype(np.float64), Z.astype(np.float64))
    assert to_np(order).tolist() == want_o.tolist()
    assert to_np(srt).tolist() == want_s.tolist()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_snap_fallback_when_candidates_taken(ctx, C, prec):
    g = np.random.default_rng(3)
    X = g.standard_normal((300, 6)).astype(np.float32)
    Z = np.repeat(g.standard_normal((2, 6)), [12, 5], axis=0).astype(np.float32)
    order, _ = C.cabs_snap(ctx, dev(X), dev(Z), prec=prec)
    want_o, _ = o.snap(X.astype(np.float64), Z.astype(np.float64))
    assert to_np(order).tolist() == want_o.tolist()
    assert len(set(to_np(order).tolist())) == Z.shape[0]


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("m,n,k,core", [(1000, 700, 256, "pinv"), (777, 1333, 200, "stabilized"),
                                        (300, 129, 65, "pinv"), (5000, 257, 33, "stabilized"), (130, 300, 8, "pinv"),
                                        (100, 90, 40, "pinv")])
def test_tc_extrapolation_matches_fp64(ctx, C, prec, m, n, k, core):
    """The extrapolation products a = C V_w, b = R^T U_w of the sketching
    routine (Section 4.1) on the tensor cores (three TF32 products, BF16 and
    TF32 modes): U = a N_c^-1, V = b N_r^-1 and S against the same products
    in FP64 from the GPU's own V_w, U_w, to 2e-5 per column (the FP32
    CUDA-core path is held to the same bar). Row counts are not multiples of
    the 128-row tile (100 and 90 fill less than one), and k = 65, 33 exercise
    widths that are not multiples of 4."""
    g = np.random.default_rng(m + n + k)
    Cm = (g.standard_normal((m, k)) * g.uniform(0.1, 10.0, size=k)).astype(np.float32)
    Rt = (g.standard_normal((n, k)) * g.uniform(0.1, 10.0, size=k)).astype(np.float32)
    W = Cm[:k].astype(np.float64)  # FP64, as the routine takes it (the FP32 values)
    res = {}
    for pr in (prec, "fp32"):
        out = C.cabs_sketching(ctx, dev(Cm), dev(Rt), dev(W), m, n, prec=pr, core=core, trunc_rtol=k * 2.0 ** -24)
        torch.cuda.synchronize()
        r = int(out["rank"].item())
        Uw, Vw, sig = (out[x].cpu().numpy() for x in ("Uw", "Vw", "sig"))
        a = Cm.astype(np.float64) @ Vw
        b = Rt.astype(np.float64) @ Uw
        nc, nr = np.linalg.norm(a, axis=0), np.linalg.norm(b, axis=0)
        S_ref = np.zeros(k)
        S_ref[:r] = sig[:r] * np.sqrt(m * n) / k if core == "stabilized" else nc[:r] * nr[:r] / sig[:r]
        U, V, S = out["out1"].cpu().numpy(), out["out2"].cpu().numpy(), out["S"].cpu().numpy()
        eu = np.linalg.norm(U[:, :r] - a[:, :r] / nc[:r], axis=0).max()
        ev = np.linalg.norm(V[:, :r] - b[:, :r] / nr[:r], axis=0).max()
        es = np.abs(S[:r] / S_ref[:r] - 1).max()
        assert np.all(U[:, r:] == 0) and np.all(V[:, r:] == 0) and np.all(S[r:] == 0)
        res[pr] = (eu, ev, es)
        assert max(eu, ev, es) <= 2e-5, (pr, eu, ev, es)
