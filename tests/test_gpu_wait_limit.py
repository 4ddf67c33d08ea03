"""Bounded device-side waits, made to run out on purpose without faulting
the GPU: the grid barriers of the cooperative kernels (the FP64 refinement of
the core SVD, the snap's greedy walk) take their poll limit from
cabs_set_wait_limit. At a limit of 0 the first CTA to reach a barrier gives up
at its first unsuccessful poll, every CTA leaves the kernel, and bit 2 of the
sketch's diagnostics status reports it. Afterwards, at the default limit, the
same context computes the same sketch as before, bit for bit.

Nothing here traps, faults or spins without a bound: a barrier that gives up
returns, and every later index the sketch uses is clamped by the gathers.
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


def sketch(C, ctx, src, m, n):
    p = C.make_params(m, n, 20, iters=5, seed=1607, prec="fp64", core="pinv")
    sk = C.cabs_sketch(ctx, src, p)
    torch.cuda.synchronize()
    return sk


def test_grid_barrier_gives_up_and_context_recovers(ctx, C):
    A = synth.plain_lowrank()
    m, n = A.shape
    src = C.dense_source(torch.from_numpy(A).cuda())
    ref = sketch(C, ctx, src, m, n)
    assert ref.diag().status == 0
    want = [t.cpu().numpy().copy() for t in (ref.rows, ref.cols, ref.U, ref.S, ref.V)]
    try:
        C.cabs_set_wait_limit(ctx, 0)
        bad = sketch(C, ctx, src, m, n)  # returns: nothing waits without a bound
        assert bad.diag().status & 4, bad.diag().status
    finally:
        C.cabs_set_wait_limit(ctx, -1)
    again = sketch(C, ctx, src, m, n)
    assert again.diag().status == 0
    got = [t.cpu().numpy() for t in (again.rows, again.cols, again.U, again.S, again.V)]
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
