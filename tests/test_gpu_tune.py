"""Launch-shape tuning through the C ABI: every cabs_tune choice leaves the
sketch bit-identical (the knobs only move work between threads and CTAs),
the table round-trips through its cache file, and cabs_autotune fills it
from timed trials on an uneven batch whose tuned batched run (lanes = 0)
still equals each member run alone.
"""
import itertools
import os
import tempfile

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


def outputs(sk):
    return [t.cpu().numpy().copy() for t in (sk.U, sk.S, sk.V, sk.rows, sk.cols, sk.pilot_rows)]


@pytest.mark.parametrize("prec,k", [("bf16", 100), ("tf32", 200), ("fp32", 64), ("fp64", 40)])
def test_every_launch_shape_gives_the_same_sketch(ctx, C, prec, k):
    A = synth.decaying_lowrank_host(3001, 1999, rank=128, seed=5)[0]
    src = C.dense_source(torch.from_numpy(A if prec != "fp64" else A.astype(np.float64)).cuda())
    p = C.make_params(3001, 1999, k, iters=4, seed=9, prec=prec, core="stabilized", trunc_rtol=k * 2.0 ** -24,
                      err_samples=0)
    C.cabs_tune_set(ctx, p, None)
    base = C.cabs_sketch(ctx, src, p)
    torch.cuda.synchronize()
    want = outputs(base) + [base.err.cpu().numpy().copy()]
    tns = (2, 4) if prec == "fp64" else (2, 4, 8)
    bns = (128, 256) if prec in ("bf16", "tf32") else (0,)
    try:
        for tn, gr, bn in itertools.product(tns, (2, 4, 8), bns):
            C.cabs_tune_set(ctx, p, dict(extrap_tn=tn, gather_rows=gr, assign_bn=bn))
            assert C.cabs_tune_get(ctx, p) == (dict(extrap_tn=tn, gather_rows=gr, assign_bn=bn), True)
            sk = C.cabs_sketch(ctx, src, p)
            torch.cuda.synchronize()
            got = outputs(sk) + [sk.err.cpu().numpy()]
            for g, w in zip(got, want):
                assert np.array_equal(g, w), (tn, gr, bn)
    finally:
        C.cabs_tune_set(ctx, p, None)


def test_invalid_shapes_rejected(ctx, C):
    p = C.make_params(1000, 1000, 32, prec="fp64")
    for bad in (dict(extrap_tn=3), dict(gather_rows=16), dict(assign_bn=64), dict(extrap_tn=8)):
        with pytest.raises(C.CabsError) as e:
            C.cabs_tune_set(ctx, p, bad)
        assert e.value.status == C.CABS_EINVAL


def batch(C, count=14, seed=3):
    specs = synth.batched_specs(count, seed=seed, lo=1000, hi=6000, k_lo=16, k_hi=128)
    srcs, params, keep = [], [], []
    for i, s in enumerate(specs):
        A = synth.decaying_lowrank_device(s["m"], s["n"], rank=s["rank"], seed=100 + i, noise_fp32=True)[0]
        keep.append(A)
        srcs.append(C.dense_source(A))
        params.append(C.make_params(s["m"], s["n"], s["k"], iters=5, seed=40 + i, prec="bf16", core="stabilized",
                                    trunc_rtol=s["k"] * 2.0 ** -24, err_samples=0))
    outs = [C.alloc_result(p) for p in params]
    offs, tot = C.batched_layout(srcs, params)
    ws = torch.empty(tot + 512, dtype=torch.uint8, device="cuda")
    return srcs, params, outs, offs, ws, keep


def test_autotune_fills_table_and_tuned_batch_matches_alone(ctx, C):
    srcs, params, outs, offs, ws, keep = batch(C)
    lanes = C.cabs_autotune(ctx, srcs, params, outs, ws, offs)
    assert lanes in (4, 8, 12, 16)
    for p in params:
        shape, found = C.cabs_tune_get(ctx, p)
        assert found
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "shapes.txt")
        C.cabs_tune_save(ctx, path)
        text = open(path).read()
        assert f"lanes {lanes}" in text
        ctx2 = C.Context(0)
        C.cabs_tune_load(ctx2, path)
        for p in params:
            assert C.cabs_tune_get(ctx2, p) == C.cabs_tune_get(ctx, p)
        # tuned batch (lanes = 0: the autotuner's lanes) against each member alone
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            C.cabs_sketch_batched(ctx2, srcs, params, outs, ws, offs, lanes=0, use_graph=True, stream=stream)
        torch.cuda.synchronize()
        got = [outputs(o) + [o.err.cpu().numpy().copy()] for o in outs]
        for i, (s, p) in enumerate(zip(srcs, params)):
            alone = C.cabs_sketch(ctx2, s, p)
            torch.cuda.synchronize()
            for g, w in zip(got[i], outputs(alone) + [alone.err.cpu().numpy()]):
                assert np.array_equal(g, w), i
        open(path, "w").write("bucket 9 1 1 2 2 2\n")
        with pytest.raises(C.CabsError):
            C.cabs_tune_load(ctx2, path)
