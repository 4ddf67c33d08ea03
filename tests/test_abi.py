"""The C-ABI library loads and exports what include/cabs.h declares; the
ctypes structures match the C layout; argument validation works on the host
(no GPU needed)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_1607_07395_gb300 import cabs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cabs.h")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(cabs.LIB_PATH):
        from paper_1607_07395_gb300 import build
        build.build()
    return cabs.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cabs_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(L, nm), nm
    assert sorted(cabs.exported_names()) == names
    out = subprocess.run(["nm", "-D", "--defined-only", cabs.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln and ln.split()[-1].startswith("cabs_")}
    assert exported == set(names)


def test_struct_layout_matches_c():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "cabs.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("cabs_source %zu\ncabs_params %zu\ncabs_diag %zu\ncabs_result %zu\n", sizeof(cabs_source),
         sizeof(cabs_params), sizeof(cabs_diag), sizeof(cabs_result));
  printf("cabs_cur_params %zu\ncabs_cur_result %zu\n", sizeof(cabs_cur_params), sizeof(cabs_cur_result));
  printf("cabs_tune %zu\n", sizeof(cabs_tune));
  F(cabs_tune, gather_rows) F(cabs_tune, assign_bn) F(cabs_tune, reserved)
  F(cabs_cur_params, kt) F(cabs_cur_params, seed) F(cabs_cur_params, prec) F(cabs_cur_params, trunc_rtol)
  F(cabs_cur_result, Ustar) F(cabs_cur_result, rows_t) F(cabs_cur_result, ranks)
  F(cabs_source, lda) F(cabs_source, X) F(cabs_source, sigma) F(cabs_source, row_ptr) F(cabs_source, nnz)
  F(cabs_params, seed) F(cabs_params, upsilon_pow) F(cabs_params, trunc_rtol) F(cabs_params, flags)
  F(cabs_params, err_samples) F(cabs_params, err_seed)
  F(cabs_diag, e_rows) F(cabs_diag, e_follow_cols) F(cabs_diag, refine_final) F(cabs_diag, reserved) F(cabs_result, diag) F(cabs_result, err)
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        lines = dict(ln.rsplit(" ", 1) for ln in subprocess.run([exe], capture_output=True, text=True,
                                                                check=True).stdout.split("\n") if ln)
    for name, cls in [("cabs_source", cabs.cabs_source), ("cabs_params", cabs.cabs_params),
                      ("cabs_diag", cabs.cabs_diag), ("cabs_result", cabs.cabs_result),
                      ("cabs_cur_params", cabs.cabs_cur_params), ("cabs_cur_result", cabs.cabs_cur_result),
                      ("cabs_tune", cabs.cabs_tune)]:
        assert int(lines[name]) == C.sizeof(cls), name
    for key, val in lines.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(cabs, t), f).offset == int(val), key


def _src():
    return cabs.cabs_source(kind=cabs.SRC_DENSE, A=0x1000, lda=1500, a_is_f64=1)


def test_workspace_size_and_validation_on_host(L):
    p = cabs.make_params(2000, 1500, 20)
    n = C.c_size_t()
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(p), C.byref(n)) == cabs.CABS_OK
    assert n.value > (2000 + 1500) * 20 * 8 * 2
    small = n.value
    p2 = cabs.make_params(2000, 1500, 20, prec="fp32")
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(p2), C.byref(n)) == cabs.CABS_OK
    assert n.value < small
    bad = [cabs.make_params(2000, 1500, 1501), cabs.make_params(2000, 1500, 20, k2=21),
           cabs.make_params(2000, 1500, 257), cabs.make_params(2000, 1500, 20, iters=65),
           cabs.make_params(0, 1500, 1), cabs.make_params(2000, 1500, 20, prec=7)]
    for b in bad:
        assert L.cabs_workspace_size(C.byref(_src()), C.byref(b), C.byref(n)) == cabs.CABS_EINVAL
        assert L.cabs_last_error(None)
    s = _src()
    s.lda = 1499
    assert L.cabs_workspace_size(C.byref(s), C.byref(p), C.byref(n)) == cabs.CABS_EINVAL
    r = cabs.cabs_source(kind=cabs.SRC_RBF, X=0x1000, Y=0x2000, d=65, sigma=1.0)
    assert L.cabs_workspace_size(C.byref(r), C.byref(p), C.byref(n)) == cabs.CABS_EINVAL
    r.d, r.sigma = 16, 0.0
    assert L.cabs_workspace_size(C.byref(r), C.byref(p), C.byref(n)) == cabs.CABS_EINVAL


def test_error_request_on_host(L):
    """CABS_FLAG_ERROR adds the error's workspace; bad requests are refused."""
    n0, n1, n2 = C.c_size_t(), C.c_size_t(), C.c_size_t()
    p = cabs.make_params(2000, 1500, 20, prec="fp32")
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(p), C.byref(n0)) == cabs.CABS_OK
    pe = cabs.make_params(2000, 1500, 20, prec="fp32", err_samples=0)
    assert pe.flags == cabs.FLAG_ERROR
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(pe), C.byref(n1)) == cabs.CABS_OK
    e = C.c_size_t()
    assert L.cabs_error_workspace_size(C.byref(_src()), C.byref(p), 0, C.byref(e)) == cabs.CABS_OK
    assert n1.value >= n0.value + e.value - 256
    ps = cabs.make_params(2000, 1500, 20, prec="fp32", err_samples=10 ** 6)
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(ps), C.byref(n2)) == cabs.CABS_OK
    bad = cabs.make_params(2000, 1500, 20, flags=32)  # no such flag
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(bad), C.byref(n0)) == cabs.CABS_EINVAL
    both = cabs.make_params(2000, 1500, 20, flags=cabs.FLAG_HARD_THRESHOLD | cabs.FLAG_LEVERAGE)
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(both), C.byref(n0)) == cabs.CABS_EINVAL
    for fl in (cabs.FLAG_LEVERAGE, cabs.FLAG_SVD_FORM):
        assert L.cabs_workspace_size(C.byref(_src()), C.byref(cabs.make_params(2000, 1500, 20, flags=fl)),
                                     C.byref(n2)) == cabs.CABS_OK
        assert n2.value > n0.value
    neg = cabs.make_params(2000, 1500, 20, err_samples=0)
    neg.err_samples = -1
    assert L.cabs_workspace_size(C.byref(_src()), C.byref(neg), C.byref(n0)) == cabs.CABS_EINVAL


def test_null_arguments_rejected(L):
    p = cabs.make_params(100, 90, 10)
    assert L.cabs_workspace_size(None, C.byref(p), None) == cabs.CABS_EINVAL
    assert L.cabs_sketch(None, C.byref(_src()), C.byref(p), None, 0, None, None) == cabs.CABS_EINVAL
    assert L.cabs_draw_indices(None, 1, 0, 10, 3, None, None, None) == cabs.CABS_EINVAL
    assert L.cabs_create(None, 0) == cabs.CABS_EINVAL


def test_no_cpu_fallback_without_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert L.cabs_create(C.byref(h), 0) == cabs.CABS_ECUDA


def test_step_workspace_sizes_validate_on_host(L):
    """Every per-step workspace query answers on the host, grows with its
    problem, and refuses what its compute call would refuse."""
    n, n2 = C.c_size_t(), C.c_size_t()
    OK, BAD = cabs.CABS_OK, cabs.CABS_EINVAL
    f64, bf16 = cabs.PREC_FP64, cabs.PREC_BF16
    # sketching routine: 1 <= k <= min(m, n, 256)
    assert L.cabs_sketching_workspace_size(2000, 1500, 20, f64, C.byref(n)) == OK and n.value > 0
    assert L.cabs_sketching_workspace_size(20000, 1500, 20, f64, C.byref(n2)) == OK and n2.value > n.value
    for m_, n_, k_, p_ in [(2000, 1500, 0, f64), (2000, 1500, 257, f64), (10, 1500, 11, f64), (2000, 1500, 20, 7)]:
        assert L.cabs_sketching_workspace_size(m_, n_, k_, p_, C.byref(n)) == BAD, (m_, n_, k_, p_)
    # k-means: 1 <= d, k2 <= 256, k2 <= M, 0 <= iters <= 64
    assert L.cabs_kmeans_workspace_size(5000, 64, 64, 5, bf16, C.byref(n)) == OK and n.value > 0
    assert L.cabs_kmeans_workspace_size(50000, 64, 64, 5, bf16, C.byref(n2)) == OK and n2.value > n.value
    for args in [(5000, 0, 64, 5, bf16), (5000, 257, 64, 5, bf16), (5000, 64, 257, 5, bf16), (10, 64, 11, 5, bf16),
                 (5000, 64, 64, 65, bf16), (5000, 64, 64, -1, bf16), (5000, 64, 64, 5, 7), (0, 64, 1, 5, bf16)]:
        assert L.cabs_kmeans_workspace_size(*args, C.byref(n)) == BAD, args
    # snap: the same bounds on M, d, k2
    assert L.cabs_snap_workspace_size(5000, 64, 64, bf16, C.byref(n)) == OK and n.value > 0
    for args in [(5000, 257, 64, bf16), (5000, 64, 0, bf16), (10, 64, 11, bf16), (5000, 64, 64, -1)]:
        assert L.cabs_snap_workspace_size(*args, C.byref(n)) == BAD, args
    # threshold: 1 <= M < 2^31
    assert L.cabs_threshold_workspace_size(5000, C.byref(n)) == OK and n.value > 0
    assert L.cabs_threshold_workspace_size(0, C.byref(n)) == BAD
    assert L.cabs_threshold_workspace_size(2 ** 31, C.byref(n)) == BAD
    # orthogonalisation: 1 <= k <= 256
    assert L.cabs_orthogonalize_workspace_size(2000, 1500, 20, f64, C.byref(n)) == OK and n.value > 0
    for args in [(2000, 1500, 0, f64), (2000, 1500, 257, f64), (0, 1500, 20, f64), (2000, 1500, 20, 9)]:
        assert L.cabs_orthogonalize_workspace_size(*args, C.byref(n)) == BAD, args
    # Sketch-CUR: 1 <= kb, kt <= min(m, n, 256)
    cp = cabs.make_cur_params(2000, 1500, 20, 60)
    assert L.cabs_sketch_cur_workspace_size(C.byref(_src()), C.byref(cp), C.byref(n)) == OK and n.value > 0
    for kb, kt in [(0, 60), (20, 257), (20, 0)]:
        bad = cabs.make_cur_params(2000, 1500, kb, kt)
        assert L.cabs_sketch_cur_workspace_size(C.byref(_src()), C.byref(bad), C.byref(n)) == BAD, (kb, kt)
    for fn in ("cabs_sketching_workspace_size", "cabs_threshold_workspace_size"):
        args = (2000, 1500, 20, f64) if fn.startswith("cabs_sketching") else (5000,)
        assert getattr(L, fn)(*args, None) == BAD
