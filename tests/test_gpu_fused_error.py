"""The relative error computed inside the sketch (CABS_FLAG_ERROR, Section 5)
must equal, bit for bit, what cabs_error returns for the same result, samples
and seed: the same kernels reduce in the same fixed order, and the final
sqrt(num / den) is correctly rounded on both sides. Also checked: the error
inside a batched graph and in the serving loop, and the host-side refusals."""
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
    assert torch.cuda.is_available()
    return C.Context(0)


def cases(C):
    out = []
    for i, (m, n, k, prec, core, samples) in enumerate([
            (2000, 1500, 20, "fp64", "pinv", 0),          # exact, FP64 residual
            (3000, 1700, 48, "fp32", "stabilized", 0),    # exact, FP32 residual on CUDA cores
            (5000, 3100, 96, "bf16", "stabilized", 0),    # exact, BF16 tensor-core residual
            (4100, 2600, 64, "tf32", "stabilized", 0),    # exact, TF32 tensor-core residual
            (3000, 1700, 48, "fp32", "stabilized", 50000)]):  # sampled on a dense source
        A, _, _, _ = synth.decaying_lowrank_host(m, n, rank=min(80, 2 * k), seed=40 + i,
                                                 dtype=np.float64 if prec == "fp64" else np.float32)
        out.append((C.dense_source(torch.from_numpy(A).cuda()), m, n, k, prec, core, samples))
    X, Y, sig = synth.rbf_mixture(6000, 5000, d=16, components=20, seed=5)
    out.append((C.rbf_source(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), sig), 6000, 5000, 64,
                "bf16", "pinv", 200000))
    return out


@pytest.mark.parametrize("i", range(6))
def test_fused_error_equals_cabs_error(ctx, C, i):
    src, m, n, k, prec, core, samples = cases(C)[i]
    p = C.make_params(m, n, k, iters=4, seed=900 + i, prec=prec, core=core, err_samples=samples, err_seed=77)
    sk = C.cabs_sketch(ctx, src, p)
    fused = float(sk.err.cpu().item())
    q = C.make_params(m, n, k, iters=4, seed=900 + i, prec=prec, core=core)
    alone = C.cabs_sketch(ctx, src, q)
    for a, b in zip((sk.U, sk.S, sk.V, sk.rows, sk.cols), (alone.U, alone.S, alone.V, alone.rows, alone.cols)):
        assert torch.equal(a, b)  # the flag changes nothing else
    ref = C.cabs_error(ctx, src, q, alone, samples=samples, seed=77)
    assert fused == ref and 0.0 <= fused < float("inf"), (fused, ref)


def test_fused_error_in_batched_graph(ctx, C):
    cs = cases(C)
    srcs, params = [], []
    for i, (src, m, n, k, prec, core, samples) in enumerate(cs):
        srcs.append(src)
        params.append(C.make_params(m, n, k, iters=4, seed=950 + i, prec=prec, core=core, err_samples=samples,
                                    err_seed=5))
    alone = []
    for src, p in zip(srcs, params):
        alone.append(float(C.cabs_sketch(ctx, src, p).err.cpu().item()))
    offs, tot = C.batched_layout(srcs, params)
    ws = torch.empty(tot + 512, dtype=torch.uint8, device="cuda")
    outs = [C.alloc_result(p) for p in params]
    stream = torch.cuda.Stream()
    for rep in range(2):
        for o in outs:
            o.err.fill_(-1.0)
        with torch.cuda.stream(stream):
            C.cabs_sketch_batched(ctx, srcs, params, outs, ws, offs, lanes=3, use_graph=True, stream=stream)
        stream.synchronize()
        assert [float(o.err.cpu().item()) for o in outs] == alone, rep


def test_fused_error_refusals(ctx, C):
    src, m, n, k, prec, core, samples = cases(C)[1]
    p = C.make_params(m, n, k, prec=prec, err_samples=0)
    sk = C.alloc_result(p)
    sk.result.err = None
    with pytest.raises(C.CabsError) as e:
        C.cabs_sketch(ctx, src, p, out=sk)
    assert e.value.status == C.CABS_EINVAL
    rsrc = cases(C)[5][0]
    pr = C.make_params(6000, 5000, 32, prec="fp32", err_samples=0)  # exact error of an implicit matrix
    with pytest.raises(C.CabsError) as e:
        C.cabs_sketch(ctx, rsrc, pr)
    assert e.value.status == C.CABS_EINVAL
