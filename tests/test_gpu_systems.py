"""Batched launch and the continuous-batching serving loop: every result must
be bit-identical to the same sketch run alone with cabs_sketch (the kernels
use no float atomics and reduce in fixed orders). Failures in the serving
loop are injected on the host (bad requests, a too-small arena, unknown
tickets); nothing faults the GPU."""
import threading
import time

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


def members(C):
    out = []
    for i, (m, n, k, prec, core) in enumerate([(1500, 1100, 24, "fp32", "stabilized"), (3000, 900, 64, "bf16", "stabilized"),
                                               (1200, 2500, 100, "fp32", "pinv"), (2000, 1500, 20, "fp64", "pinv"),
                                               (5000, 3000, 128, "bf16", "stabilized")]):
        A, _, _, _ = synth.decaying_lowrank_host(m, n, rank=min(60, k * 2), seed=10 + i,
                                                 dtype=np.float64 if prec == "fp64" else np.float32)
        Ad = torch.from_numpy(A).cuda()
        out.append((C.dense_source(Ad), C.make_params(m, n, k, iters=4, seed=100 + i, prec=prec, core=core)))
    X, Y, sig = synth.rbf_mixture(4000, 3500, d=16, components=20, seed=3)
    out.append((C.rbf_source(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), sig),
                C.make_params(4000, 3500, 48, iters=5, seed=7, prec="fp32")))
    # the Section 5 variants, the SVD form and a sparse source with its exact error
    A, _, _, _ = synth.decaying_lowrank_host(2500, 1800, rank=50, seed=21)
    Ad = torch.from_numpy(A).cuda()
    out.append((C.dense_source(Ad), C.make_params(2500, 1800, 40, iters=3, seed=31, prec="bf16",
                                                  flags=C.FLAG_SVD_FORM)))
    out.append((C.dense_source(Ad), C.make_params(2500, 1800, 40, 24, iters=3, seed=32, prec="fp32",
                                                  flags=C.FLAG_LEVERAGE)))
    ip, ix, v = synth.sparse_lowrank(3000, 2500, 0.02, rank=8, seed=5)
    csr = C.csr_source(torch.from_numpy(ip).cuda(), torch.from_numpy(ix).cuda(), torch.from_numpy(v).cuda())
    out.append((csr, C.make_params(3000, 2500, 48, iters=4, seed=33, prec="bf16", flags=C.FLAG_HARD_THRESHOLD,
                                   err_samples=0)))
    return out


def host(sk):
    return [t.cpu().numpy() for t in (sk.U, sk.S, sk.V, sk.rows, sk.cols, sk.pilot_rows, sk.pilot_cols, sk.err)]


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("use_graph,lanes", [(False, 1), (False, 3), (True, 3), (True, 4)])
def test_batched_bit_identical_to_alone(ctx, C, use_graph, lanes):
    mem = members(C)
    alone = []
    for src, p in mem:
        alone.append(host(C.cabs_sketch(ctx, src, p)))
    torch.cuda.synchronize()
    srcs, params = [s for s, _ in mem], [p for _, p in mem]
    offs, tot = C.batched_layout(srcs, params)
    ws = torch.empty(tot + 512, dtype=torch.uint8, device="cuda")
    outs = [C.alloc_result(p) for p in params]
    stream = torch.cuda.Stream()
    for rep in range(2):  # the second run replays the captured graph
        for o in outs:
            o.U.zero_()
        with torch.cuda.stream(stream):
            C.cabs_sketch_batched(ctx, srcs, params, outs, ws, offs, lanes=lanes, use_graph=use_graph, stream=stream)
        stream.synchronize()
        for i, o in enumerate(outs):
            assert same(host(o), alone[i]), (rep, i)


def test_serving_mix_equals_alone_and_overlaps(ctx, C):
    base = members(C)
    nb = len(base)
    mem = base * 3
    alone = {}
    for i, (src, p) in enumerate(base):
        alone[i] = host(C.cabs_sketch(ctx, src, p))
    torch.cuda.synchronize()
    # an arena that cannot hold every request at once: admission must queue
    need = max(C.cabs_workspace_size(s, p) for s, p in mem) * 3
    srv = C.Server(ctx, arena_bytes=need, max_slots=4)
    try:
        tickets = []

        def client():
            for i, (src, p) in enumerate(mem):
                tickets.append((i % nb, srv.submit(src, p)))
                time.sleep(0.0005)

        th = threading.Thread(target=client)
        th.start()
        th.join()
        lat, ivals = [], []
        for idx, t in tickets:
            r = None
            for _ in range(2000):
                r = srv.poll(t, timeout_ms=50)
                if r is not None:
                    break
            assert r is not None, "request never finished"
            res, ms = r
            lat.append(ms)
            ivals.append(srv.times(t))
            U, S, V, rows, cols = C.result_tensors(res, mem[idx][1])
            got = [x.cpu().numpy() for x in (U, S, V, rows, cols)]
            assert same(got, alone[idx][:5]), idx
            srv.release(t)
        assert all(x > 0 for x in lat)
        assert all(0 <= a <= b for a, b in ivals)
        # at least two requests had work on the GPU at the same time
        ivals.sort()
        assert any(ivals[j][0] < ivals[i][1] for i in range(len(ivals)) for j in range(i + 1, len(ivals))), ivals
    finally:
        srv.stop()


def test_serving_host_side_faults(ctx, C):
    src, p = members(C)[0]
    small = C.Server(ctx, arena_bytes=64 << 10, max_slots=2)
    try:
        with pytest.raises(C.CabsError) as e:
            small.submit(src, p)                       # footprint exceeds the arena
        assert e.value.status == C.CABS_ENOMEM
        bad = C.make_params(100, 100, 200)             # k > min(m, n)
        with pytest.raises(C.CabsError) as e:
            small.submit(src, bad)
        assert e.value.status == C.CABS_EINVAL
        with pytest.raises(C.CabsError) as e:
            small.poll(987654, timeout_ms=0)
        assert e.value.status == C.CABS_ENOTFOUND
    finally:
        small.stop()
    srv = C.Server(ctx, arena_bytes=C.cabs_workspace_size(src, p) * 4, max_slots=1)
    try:
        t = srv.submit(src, p)
        r = None
        for _ in range(2000):
            r = srv.poll(t, timeout_ms=50)
            if r is not None:
                break
        assert r is not None
        with pytest.raises(C.CabsError) as e:
            srv.release(t + 1)
        assert e.value.status == C.CABS_ENOTFOUND
        srv.release(t)
    finally:
        srv.stop()
