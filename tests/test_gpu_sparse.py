"""GPU parity on sparse inputs in compressed rows (CABS_SRC_CSR; Table 1's
sparse data) through the C ABI against the FP64 oracle's CSR source.

Bars: gathers bit-exact (they copy stored values); indices of whole sketches
bit-exact in FP64 with factors within 1e-10 of the oracle's; the exact error
by the linear-cost identity within 1e-9 of the oracle's dense definition in
FP64. In FP32 the identity subtracts FP64 sums whose inputs carry the FP32
rounding of U, V and of each k-term dot product (about 2^-24 sqrt(k)
relative), so the squared error agrees to 2e-6 of |A|^2 + |L|^2 and the
error to that over twice itself.
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


def make(C, m, n, density, rank, seed, f64=False):
    ip, ix, v = synth.sparse_lowrank(m, n, density, rank=rank, seed=seed)
    vals = v.astype(np.float64) if f64 else v
    src = C.csr_source(torch.from_numpy(ip).cuda(), torch.from_numpy(ix).cuda(), torch.from_numpy(vals).cuda())
    return src, o.CSRSource(ip, ix, vals, n)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m,n,density,kr,kc", [(2000, 1500, 0.02, 40, 40), (777, 1300, 0.005, 64, 17),
                                                (300, 5000, 0.1, 1, 200)])
def test_csr_gather_bit_exact(ctx, C, prec, m, n, density, kr, kc):
    src, ref = make(C, m, n, density, 5, m + n, f64=(prec == "fp64"))
    g = np.random.default_rng(1)
    rows = np.sort(g.choice(m, kr, replace=False)).astype(np.int32)
    cols = np.sort(g.choice(n, kc, replace=False)).astype(np.int32)
    Cm, Rt, W = C.cabs_gather(ctx, src, m, n, torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda(), prec=prec)
    torch.cuda.synchronize()
    Cw, Rw, Ww = ref.gather(rows, cols)
    assert np.array_equal(Cm.double().cpu().numpy(), Cw)
    assert np.array_equal(Rt.double().cpu().numpy(), Rw)
    assert np.array_equal(W.cpu().numpy(), Ww)


@pytest.mark.parametrize("follow", ["kmeans", "threshold", "leverage"])
@pytest.mark.parametrize("mode", ["pinv", "stabilized"])
def test_sparse_fp64_sketch_matches_oracle(ctx, C, follow, mode):
    # At low density many embedding rows coincide (rows with the same few
    # stored entries among the pilot columns), and the k-means and the snap
    # then decide exact ties by rounding order; any tie-break is valid. The
    # k-means variant is compared where rows are distinct (density 0.5).
    density = 0.5 if follow == "kmeans" else 0.05
    src, ref_src = make(C, 2000, 1500, density, 10, 7, f64=True)
    flags = {"kmeans": C.FLAG_FOLLOW_ERR, "threshold": C.FLAG_HARD_THRESHOLD, "leverage": C.FLAG_LEVERAGE}[follow]
    p = C.make_params(2000, 1500, 40, 30, iters=5, seed=1607, prec="fp64", core=mode, flags=flags, err_samples=0)
    sk = C.cabs_sketch(ctx, src, p)
    torch.cuda.synchronize()
    ref = o.cabs(ref_src, 40, 30, iters=5, seed=1607, mode=mode, follow=follow)
    assert sk.pilot_rows.tolist() == ref.pilot_rows.tolist()
    assert sk.rows.tolist() == ref.rows.tolist()
    assert sk.cols.tolist() == ref.cols.tolist()
    U, S, V = sk.U.cpu().numpy(), sk.S.cpu().numpy(), sk.V.cpu().numpy()
    want = (ref.final.U * ref.final.S) @ ref.final.V.T
    assert np.linalg.norm((U * S) @ V.T - want) <= 1e-10 * max(np.linalg.norm(want), 1e-300)
    e_ref = o.rel_fro_error_dense(ref_src.dense(), ref.final.U, ref.final.S, ref.final.V)
    assert abs(sk.err.item() - e_ref) <= 1e-9 * e_ref


def upload(C, p, F):
    """A result holding the oracle's factors (U, S, V), as the error call takes them."""
    U, S, V = F
    dt = torch.float64 if p.prec == C.PREC_FP64 else torch.float32
    r = C.alloc_result(p, "cuda")
    r.U.copy_(torch.from_numpy(np.ascontiguousarray(U)).to(dt))
    r.S.copy_(torch.from_numpy(np.ascontiguousarray(S)))
    r.V.copy_(torch.from_numpy(np.ascontiguousarray(V)).to(dt))
    return r


def test_sparse_exact_error_fp32(ctx, C):
    """The linear-cost exact error on the oracle's sketch factors (rounded to
    FP32, as the FP32 mode holds them) against the dense definition."""
    src, ref_src = make(C, 4000, 3000, 0.01, 10, 11)
    ref = o.cabs(ref_src, 64, iters=5, seed=3, mode="stabilized")
    F = [x.astype(np.float32).astype(np.float64) for x in (ref.final.U, ref.final.V)]
    U, V, S = F[0], F[1], ref.final.S
    p = C.make_params(4000, 3000, 64, iters=5, seed=3, prec="fp32", core="stabilized")
    e_gpu = C.cabs_error(ctx, src, p, upload(C, p, (U, S, V)))
    A = ref_src.dense()
    e_ref = o.rel_fro_error_dense(A, U, S, V)
    a2 = np.sum(A ** 2)
    l2 = np.sum(((U * S) @ V.T) ** 2)
    tol = 2e-6 * (a2 + l2) / a2 / (2 * e_ref)
    assert abs(e_gpu - e_ref) <= tol * e_ref + 1e-12


def test_sparse_exact_error_fp64(ctx, C):
    src, ref_src = make(C, 3000, 2500, 0.02, 8, 12, f64=True)
    ref = o.cabs(ref_src, 32, iters=5, seed=9, mode="pinv")
    F = (ref.final.U, ref.final.S, ref.final.V)
    p = C.make_params(3000, 2500, 32, iters=5, seed=9, prec="fp64", core="pinv")
    e_gpu = C.cabs_error(ctx, src, p, upload(C, p, F))
    e_ref = o.rel_fro_error_dense(ref_src.dense(), *F)
    assert abs(e_gpu - e_ref) <= 1e-9 * e_ref


def test_sparse_sampled_error_fp64(ctx, C):
    src, ref_src = make(C, 3000, 2500, 0.02, 8, 13, f64=True)
    ref = o.cabs(ref_src, 32, iters=5, seed=9, mode="pinv")
    F = (ref.final.U, ref.final.S, ref.final.V)
    p = C.make_params(3000, 2500, 32, iters=5, seed=9, prec="fp64", core="pinv")
    e_gpu = C.cabs_error(ctx, src, p, upload(C, p, F), samples=200000, seed=3)
    e_ref = o.rel_fro_error_sampled(ref_src, *F, 3, 200000)
    assert abs(e_gpu - e_ref) <= 1e-10 * e_ref


def test_sparse_ratings_shape_runs(ctx, C):
    """Table 1's movie-ratings shape (27000 x 46000, 0.56 %), k = 256, BF16:
    valid indices, the hard-threshold variant too, a finite positive exact
    error and a clean SVD status."""
    ip, ix, v = synth.sparse_lowrank()
    src = C.csr_source(torch.from_numpy(ip).cuda(), torch.from_numpy(ix).cuda(), torch.from_numpy(v).cuda())
    for flags in (0, C.FLAG_HARD_THRESHOLD):
        p = C.make_params(27000, 46000, 256, iters=5, seed=1607, prec="bf16", core="stabilized", flags=flags,
                          trunc_rtol=256 * 2.0 ** -24, err_samples=0)
        sk = C.cabs_sketch(ctx, src, p)
        torch.cuda.synchronize()
        for idx, N in ((sk.rows, 27000), (sk.cols, 46000)):
            x = idx.cpu().numpy()
            assert len(set(x.tolist())) == 256 and np.all(np.diff(x) > 0) and x.min() >= 0 and x.max() < N
        assert 0.0 < sk.err.item() < float("inf") and sk.diag().status == 0
