"""cabs_error_noalloc: the error entry point for callers that cannot allocate
device memory (a framework's memory pool that forbids cudaMalloc/cudaFree
during a step, or a program that reserved all device memory up front).

It must return what cabs_error returns, call after call: its scratch is a
fixed device array shared by every call, so two calls in a row also check
that nothing left over from the first call leaks into the second. In the
TF32 and BF16 modes on a dense FP32 A, cabs_error forms the products on
tensor cores while this variant uses FP32 CUDA-core products: there it must
equal the FP32-mode value of the same factors and lie within 1e-3 relative
of cabs_error's. This file
is collected last on purpose; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from workloads import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def C():
    from paper_1607_07395_gb300 import cabs
    return cabs


@pytest.fixture(scope="module")
def ctx(C):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return C.Context(0)


def test_exact_error_matches_cabs_error_twice(ctx, C):
    A = synth.plain_lowrank()
    Ad = torch.from_numpy(A).cuda()
    src = C.dense_source(Ad)
    p = C.make_params(2000, 1500, 20, iters=5, seed=1607, prec="fp64")
    sk = C.cabs_sketch(ctx, src, p)
    want = C.cabs_error(ctx, src, p, sk)
    for _ in range(2):
        got = C.cabs_error_noalloc(ctx, src, p, sk)
        assert abs(got - want) <= 1e-9 * want, (got, want)


def test_fp32_exact_and_sampled_twice(ctx, C):
    A, _, _, _ = synth.decaying_lowrank_host(3000, 1700, rank=64, seed=3)
    Ad = torch.from_numpy(A).cuda()
    src = C.dense_source(Ad)
    p = C.make_params(3000, 1700, 48, iters=3, seed=5, prec="fp32", core="stabilized")
    sk = C.cabs_sketch(ctx, src, p)
    for samples in (0, 123457):
        want = C.cabs_error(ctx, src, p, sk, samples=samples, seed=9)
        for _ in range(2):
            got = C.cabs_error_noalloc(ctx, src, p, sk, samples=samples, seed=9)
            assert abs(got - want) <= 1e-9 * want, (samples, got, want)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_reduced_precision_exact_twice(ctx, C, prec):
    A, _, _, _ = synth.decaying_lowrank_host(3000, 1700, rank=64, seed=3)
    Ad = torch.from_numpy(A).cuda()
    src = C.dense_source(Ad)
    p = C.make_params(3000, 1700, 48, iters=3, seed=5, prec=prec, core="stabilized")
    sk = C.cabs_sketch(ctx, src, p)
    want_tc = C.cabs_error(ctx, src, p, sk)                     # tensor-core residual
    p32 = C.make_params(3000, 1700, 48, iters=3, seed=5, prec="fp32", core="stabilized")
    want_32 = C.cabs_error(ctx, src, p32, sk)                   # FP32 products, same factors
    for _ in range(2):
        got = C.cabs_error_noalloc(ctx, src, p, sk)
        assert abs(got - want_32) <= 1e-9 * want_32, (got, want_32)
        assert abs(got - want_tc) <= 1e-3 * want_tc, (got, want_tc)


def test_rbf_sampled_twice(ctx, C):
    X, Y, sig = synth.rbf_mixture(4000, 3500, d=16, components=20)
    src = C.rbf_source(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), sig)
    p = C.make_params(4000, 3500, 32, iters=4, seed=2, prec="fp32")
    sk = C.cabs_sketch(ctx, src, p)
    want = C.cabs_error(ctx, src, p, sk, samples=200000, seed=4)
    for _ in range(2):
        got = C.cabs_error_noalloc(ctx, src, p, sk, samples=200000, seed=4)
        assert abs(got - want) <= 1e-9 * want, (got, want)


def test_rows_beyond_the_scratch_are_rejected(ctx, C):
    tiny = torch.zeros(1, 1, dtype=torch.float32, device="cuda")
    src = C.dense_source(tiny)
    p = C.make_params(2_000_000, 1, 1, iters=0, prec="fp32")
    sk = C.alloc_result(C.make_params(1, 1, 1, iters=0, prec="fp32"))
    with pytest.raises(C.CabsError) as e:
        C.cabs_error_noalloc(ctx, src, p, sk)
    assert e.value.status == C.CABS_EINVAL and "1048576" in str(e.value)
