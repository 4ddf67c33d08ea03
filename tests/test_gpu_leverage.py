"""GPU parity of the leverage-score follow-up (Section 5, follow-up variant
(e)) through the C ABI against the FP64 oracle.

The follow-up indices are integers decided by FP64 keys l_i / (-ln u_i); the
GPU's leverage scores come from its own FP64 orthogonalisation (agreeing with
the oracle's to about 1e-13 relative) and its own logarithm (within an ulp).
So the indices must be identical unless the oracle's k2-th and (k2+1)-th keys
lie within 1e-9 relative of each other, which is checked and absent on these
inputs; the sketch itself then follows the FP64 factor bar (1e-10).
"""
import numpy as np
import pytest

from oracle import cabs_ref as o
from workloads import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1607_07395_gb300 import cabs
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return cabs


@pytest.fixture(scope="module")
def ctx(C):
    return C.Context(0)


def no_near_tie(P, Q, k1, k2, seed, trunc_rtol=0.0):
    X, _, Y = o.orthogonalize(P, np.ones(k1), Q, trunc_rtol)
    for F, tag in ((X, o.TAG_LEV_ROWS), (Y, o.TAG_LEV_COLS)):
        _, keys = o.weighted_sample(o.leverage_scores(F), k2, seed, tag)
        ks = np.sort(keys)[::-1]
        if k2 < len(ks):
            assert ks[k2 - 1] - ks[k2] > 1e-9 * ks[k2 - 1]


@pytest.mark.parametrize("mode", ["pinv", "stabilized"])
@pytest.mark.parametrize("k1,k2", [(20, 20), (20, 8)])
def test_plain_fp64_leverage_sketch_matches_oracle(ctx, C, mode, k1, k2):
    A = synth.plain_lowrank()
    m, n = A.shape
    Ad = torch.from_numpy(A).cuda()
    p = C.make_params(m, n, k1, k2, iters=5, seed=1607, prec="fp64", core=mode, flags=C.FLAG_LEVERAGE)
    sk = C.cabs_sketch(ctx, C.dense_source(Ad), p)
    torch.cuda.synchronize()
    ref = o.cabs(o.DenseSource(A), k1, k2, seed=1607, mode=mode, follow="leverage")
    no_near_tie(ref.P, ref.Q, k1, k2, 1607)
    assert sk.pilot_rows.tolist() == ref.pilot_rows.tolist()
    assert sk.rows.tolist() == ref.rows.tolist()
    assert sk.cols.tolist() == ref.cols.tolist()
    U, S, V = sk.U.cpu().numpy(), sk.S.cpu().numpy(), sk.V.cpu().numpy()
    want = (ref.final.U * ref.final.S) @ ref.final.V.T
    assert np.linalg.norm((U * S) @ V.T - want) <= 1e-10 * np.linalg.norm(want)
    d = sk.diag()
    assert d.rank_final == ref.final.rank and d.status == 0 and list(d.e_rows)[:5] == [0.0] * 5


def test_rbf_fp64_leverage_sketch_matches_oracle(ctx, C):
    X, Y, sig = synth.rbf_mixture(6000, 5000, d=16, components=50)
    src = C.rbf_source(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), sig)
    p = C.make_params(6000, 5000, 40, 30, seed=5, prec="fp64", core="pinv", trunc_rtol=1e-10,
                      flags=C.FLAG_LEVERAGE)
    sk = C.cabs_sketch(ctx, src, p)
    torch.cuda.synchronize()
    ref = o.cabs(o.RBFSource(X, Y, sig), 40, 30, seed=5, mode="pinv", trunc_rtol=1e-10, follow="leverage")
    no_near_tie(ref.P, ref.Q, 40, 30, 5, 1e-10)
    assert sk.rows.tolist() == ref.rows.tolist()
    assert sk.cols.tolist() == ref.cols.tolist()


def test_zero_rows_never_drawn(ctx, C):
    """Rows of A that are zero have zero leverage and are never drawn."""
    A = synth.exact_lowrank_int(3000, 2000, 6, seed=2)
    A[:1000] = 0.0
    Ad = torch.from_numpy(A).cuda()
    p = C.make_params(3000, 2000, 16, 12, seed=3, prec="fp64", flags=C.FLAG_LEVERAGE)
    sk = C.cabs_sketch(ctx, C.dense_source(Ad), p)
    torch.cuda.synchronize()
    rows = sk.rows.cpu().numpy()
    assert rows.min() >= 1000 and len(set(rows.tolist())) == 12 and np.all(np.diff(rows) > 0)
    U, S, V = sk.U.cpu().numpy(), sk.S.cpu().numpy(), sk.V.cpu().numpy()
    assert np.linalg.norm((U * S) @ V.T - A) <= 1e-9 * np.linalg.norm(A)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_reduced_precision_leverage_sketch_valid(ctx, C, prec):
    """FP32 / BF16: valid distinct sorted indices and an error close to FP64's."""
    A, _, _, _ = synth.decaying_lowrank_host(4096, 2048, rank=256, decay=30, noise_std=1e-4, seed=1607)
    src = C.dense_source(torch.from_numpy(A).cuda())
    errs = {}
    for pr in ("fp64", prec):
        p = C.make_params(4096, 2048, 128, 128, seed=1607, prec=pr, core="stabilized", flags=C.FLAG_LEVERAGE,
                          err_samples=0)
        sk = C.cabs_sketch(ctx, src, p)
        torch.cuda.synchronize()
        for idx, N in ((sk.rows, 4096), (sk.cols, 2048)):
            v = idx.cpu().numpy()
            assert len(set(v.tolist())) == 128 and np.all(np.diff(v) > 0) and v.min() >= 0 and v.max() < N
        errs[pr] = sk.err.item()
    assert abs(errs[prec] - errs["fp64"]) <= 0.05 * errs["fp64"]
