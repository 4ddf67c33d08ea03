"""GPU parity of Sketch-CUR (Section 2.2, Algorithm 1 with independent base
and target draws) through the C ABI against the FP64 oracle.

Bars: the four index draws bit-exact. U* = C_bar^+ M R_bar^+ solves a least
squares problem with a residual, whose solution moves by up to about
eps (kappa_C^2 + kappa_R^2) relative when the pseudo-inverses are perturbed at
the level eps (kappa: the condition number of the kept part of C_bar, R_bar);
the GPU reaches them through the FP64-accurate SVD of each block padded to
K x K, whose singular vectors carry exactly such an error. So U* must agree to
tol_U = 50 K 2^-52 (kappa_C^2 + kappa_R^2) relative (K = max(kb, kt); the 50
covers the constants of the two SVDs' backward errors and the four products), and the
product C U* R to tol_U |C| |U*| |R| / |A|. An exactly low-rank matrix is
recovered to 1e-9. FP32 inputs: U* is still FP64 from exact FP32 entries;
U = C U* is an FP32 product over kb terms (2^-24 sqrt(kb) relative per
entry), so the relative error of the sketch agrees with the oracle's to 1e-5.
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


def run(ctx, A, kb, kt, seed, prec, trunc_rtol=0.0):
    from paper_1607_07395_gb300 import cabs
    m, n = A.shape
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    src = cabs.dense_source(Ad)
    p = cabs.make_cur_params(m, n, kb, kt, seed=seed, prec=prec, trunc_rtol=trunc_rtol)
    out = cabs.cabs_sketch_cur(ctx, src, p)
    torch.cuda.synchronize()
    return p, src, out


def tol_u(ref, A_entries, trunc_rtol=0.0):
    """tol_U of the module docstring from the oracle's kept singular values."""
    Cbar = ref.C[ref.rows_t, :]
    Rbar = ref.Rt[ref.cols_t, :].T
    K = max(Cbar.shape[0], Cbar.shape[1])
    kap = []
    for B in (Cbar, Rbar):
        sv = np.linalg.svd(B, compute_uv=False)
        kept = sv[sv > max(trunc_rtol, K * 2.0 ** -52) * sv[0]]
        kap.append(kept[0] / kept[-1])
    return 50 * K * 2.0 ** -52 * (kap[0] ** 2 + kap[1] ** 2)


def same_indices(out, ref):
    assert out.rows_b.tolist() == ref.rows_b.tolist()
    assert out.cols_b.tolist() == ref.cols_b.tolist()
    assert out.rows_t.tolist() == ref.rows_t.tolist()
    assert out.cols_t.tolist() == ref.cols_t.tolist()


@pytest.mark.parametrize("kb,kt", [(20, 60), (20, 20), (30, 10), (1, 3), (7, 1), (64, 192)])
def test_plain_fp64_sketch_cur_matches_oracle(ctx, kb, kt):
    A = synth.plain_lowrank()
    p, src, out = run(ctx, A, kb, kt, 1607, "fp64")
    ref = o.sketch_cur(o.DenseSource(A), kb, kt, seed=1607)
    same_indices(out, ref)
    tu = tol_u(ref, A)
    Us = out.Ustar.cpu().numpy()
    assert np.linalg.norm(Us - ref.U) <= tu * np.linalg.norm(ref.U)
    got = out.U.cpu().numpy() @ out.V.cpu().numpy().T
    want = ref.C @ ref.U @ ref.Rt.T
    scale = np.linalg.norm(ref.C, 2) * np.linalg.norm(ref.U, 2) * np.linalg.norm(ref.Rt, 2)
    assert np.linalg.norm(got - want) <= tu * scale + 1e-12 * np.linalg.norm(A)
    assert np.all(out.S.cpu().numpy() == 1.0)


def test_exact_lowrank_recovered(ctx):
    A = synth.exact_lowrank_int(500, 400, 5, seed=3)
    p, src, out = run(ctx, A, 8, 24, 9, "fp64")
    ref = o.sketch_cur(o.DenseSource(A), 8, 24, seed=9)
    same_indices(out, ref)
    assert out.ranks.tolist()[:2] == [5, 5]
    got = out.U.cpu().numpy() @ out.V.cpu().numpy().T
    assert np.linalg.norm(got - A) <= 1e-9 * np.linalg.norm(A)


def test_fp32_sketch_cur_error_matches_oracle(ctx):
    from paper_1607_07395_gb300 import cabs
    A, _, _, _ = synth.decaying_lowrank_host(4096, 2048, rank=256, decay=30, noise_std=1e-4, seed=1607)
    p, src, out = run(ctx, A, 64, 192, 1607, "fp32")
    ref = o.sketch_cur(o.DenseSource(A), 64, 192, seed=1607)
    same_indices(out, ref)
    assert np.linalg.norm(out.Ustar.cpu().numpy() - ref.U) <= tol_u(ref, A) * np.linalg.norm(ref.U)
    e_ref = o.rel_fro_error_dense(A, ref.C @ ref.U, np.ones(64), ref.Rt)
    sp = cabs.make_params(4096, 2048, 64, prec="fp32")
    e_gpu = cabs.cabs_error(ctx, src, sp, out)
    assert abs(e_gpu - e_ref) <= 1e-5 * e_ref


def test_rbf_fp64_sketch_cur_error_matches_oracle(ctx):
    from paper_1607_07395_gb300 import cabs
    X, Y, sig = synth.rbf_mixture(3000, 2500, d=16, components=50)
    src = cabs.rbf_source(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), sig)
    # RBF blocks have fast-decaying spectra: a cut at 1e-4 keeps kappa <= 1e4
    p = cabs.make_cur_params(3000, 2500, 30, 90, seed=5, prec="fp64", trunc_rtol=1e-4)
    out = cabs.cabs_sketch_cur(ctx, src, p)
    torch.cuda.synchronize()
    ref = o.sketch_cur(o.RBFSource(X, Y, sig), 30, 90, seed=5, trunc_rtol=1e-4)
    same_indices(out, ref)
    tu = tol_u(ref, None, 1e-4)
    assert np.linalg.norm(out.Ustar.cpu().numpy() - ref.U) <= tu * np.linalg.norm(ref.U)
    sp = cabs.make_params(3000, 2500, 30, prec="fp64")
    e_gpu = cabs.cabs_error(ctx, src, sp, out, samples=200000, seed=3)
    e_ref = o.rel_fro_error_sampled(o.RBFSource(X, Y, sig), ref.C @ ref.U, np.ones(30), ref.Rt, 3, 200000)
    assert abs(e_gpu - e_ref) <= max(10 * tu, 1e-9) * max(e_ref, 1e-30)


def test_sketch_cur_full_width(ctx):
    """kb = 85, kt = 255 (target three times the base, the largest K) on a
    16384 x 8192 FP32 matrix: against the oracle on the same matrix."""
    from paper_1607_07395_gb300 import cabs
    A, _, _, _ = synth.decaying_lowrank_device(16384, 8192, rank=256, decay=30, noise_std=1e-4, seed=7)
    src = cabs.dense_source(A)
    p = cabs.make_cur_params(16384, 8192, 85, 255, seed=21, prec="fp32")
    out = cabs.cabs_sketch_cur(ctx, src, p)
    torch.cuda.synchronize()
    Ah = A.cpu().numpy()
    ref = o.sketch_cur(o.DenseSource(Ah), 85, 255, seed=21)
    same_indices(out, ref)
    assert np.linalg.norm(out.Ustar.cpu().numpy() - ref.U) <= tol_u(ref, Ah) * np.linalg.norm(ref.U)
    rows = np.arange(0, 16384, 97)
    got = out.U.double().cpu().numpy()[rows] @ out.V.double().cpu().numpy().T
    want = (ref.C[rows] @ ref.U) @ ref.Rt.T
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
