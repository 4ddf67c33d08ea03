"""Python binding of libcabs (include/cabs.h): argument marshalling only.

Every computation runs in libcabs.so on the GPU. Functions keep the C names;
they take torch CUDA tensors (device memory comes from torch), pass raw
pointers and the current torch stream, and raise CabsError on a non-zero
status. If the shared library is missing, loading fails loudly: there is no
CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcabs.so")

CABS_OK, CABS_EINVAL, CABS_ENOMEM, CABS_ECUDA, CABS_ETIMEOUT, CABS_EBUSY, CABS_ERANK, CABS_ENOTFOUND = range(8)
PREC_FP64, PREC_FP32, PREC_TF32, PREC_BF16 = range(4)
CORE_PINV, CORE_STABILIZED = 0, 1
SRC_DENSE, SRC_RBF, SRC_CSR = 0, 1, 2
TAG_ROWS, TAG_COLS, TAG_EVAL = 0, 1, 2
MAX_K, MAX_D, MAX_ITERS = 256, 64, 64
FLAG_FOLLOW_ERR = 1
FLAG_ERROR = 2
FLAG_HARD_THRESHOLD = 4
FLAG_SVD_FORM = 8
FLAG_LEVERAGE = 16
PRECS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "tf32": PREC_TF32, "bf16": PREC_BF16}
CORES = {"pinv": CORE_PINV, "stabilized": CORE_STABILIZED}


class CabsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libcabs status {status}: {msg}")
        self.status = status


class cabs_source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("A", C.c_void_p), ("lda", C.c_int64), ("a_is_f64", C.c_int32),
                ("X", C.c_void_p), ("Y", C.c_void_p), ("d", C.c_int32), ("sigma", C.c_float),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("nnz", C.c_int64)]


class cabs_params(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("k1", C.c_int32), ("k2", C.c_int32), ("iters", C.c_int32),
                ("seed", C.c_uint64), ("prec", C.c_int32), ("core", C.c_int32), ("upsilon_pow", C.c_float),
                ("trunc_rtol", C.c_double), ("flags", C.c_int32), ("err_samples", C.c_int64),
                ("err_seed", C.c_uint64)]


class cabs_diag(C.Structure):
    _fields_ = [("rank_pilot", C.c_int32), ("rank_final", C.c_int32), ("sweeps_pilot", C.c_int32),
                ("sweeps_final", C.c_int32), ("T_rows", C.c_int32), ("T_cols", C.c_int32), ("status", C.c_int32),
                ("rechecked", C.c_int32), ("e_rows", C.c_double * MAX_ITERS), ("e_cols", C.c_double * MAX_ITERS),
                ("e_follow_rows", C.c_double), ("e_follow_cols", C.c_double), ("snap_fallbacks", C.c_int32),
                ("refine_pilot", C.c_int32), ("refine_final", C.c_int32), ("reserved", C.c_int32)]


class cabs_result(C.Structure):
    _fields_ = [("U", C.c_void_p), ("S", C.c_void_p), ("V", C.c_void_p), ("rows", C.c_void_p),
                ("cols", C.c_void_p), ("pilot_rows", C.c_void_p), ("pilot_cols", C.c_void_p),
                ("diag", C.c_void_p), ("err", C.c_void_p)]


class cabs_tune(C.Structure):
    _fields_ = [("extrap_tn", C.c_int32), ("gather_rows", C.c_int32), ("assign_bn", C.c_int32), ("reserved", C.c_int32)]


class cabs_cur_params(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("kb", C.c_int32), ("kt", C.c_int32), ("seed", C.c_uint64),
                ("prec", C.c_int32), ("trunc_rtol", C.c_double)]


class cabs_cur_result(C.Structure):
    _fields_ = [("U", C.c_void_p), ("S", C.c_void_p), ("V", C.c_void_p), ("Ustar", C.c_void_p),
                ("rows_b", C.c_void_p), ("cols_b", C.c_void_p), ("rows_t", C.c_void_p), ("cols_t", C.c_void_p),
                ("ranks", C.c_void_p)]


_lib = None


def lib():
    """The loaded libcabs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it first (python -m paper_1607_07395_gb300.build); "
                           "libcabs has no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64, f32, f64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float, C.c_double, C.c_size_t
    P = C.POINTER
    sig = {
        "cabs_create": ([P(vp), C.c_int], i32),
        "cabs_destroy": ([vp], None),
        "cabs_last_error": ([vp], C.c_char_p),
        "cabs_version": ([], C.c_char_p),
        "cabs_workspace_size": ([P(cabs_source), P(cabs_params), P(sz)], i32),
        "cabs_sketch": ([vp, P(cabs_source), P(cabs_params), vp, sz, vp, P(cabs_result)], i32),
        "cabs_sketch_batched": ([vp, i32, P(cabs_source), P(cabs_params), vp, P(sz), P(cabs_result), i32, i32, vp],
                                i32),
        "cabs_error_workspace_size": ([P(cabs_source), P(cabs_params), i64, P(sz)], i32),
        "cabs_error": ([vp, P(cabs_source), P(cabs_params), P(cabs_result), i64, u64, vp, sz, vp, P(f64)], i32),
        "cabs_draw_indices": ([vp, u64, i32, i64, i32, vp, vp, vp], i32),
        "cabs_gather": ([vp, P(cabs_source), i64, i64, vp, i32, vp, i32, i32, vp, vp, vp, vp], i32),
        "cabs_sketching_workspace_size": ([i64, i64, i32, i32, P(sz)], i32),
        "cabs_sketching": ([vp, i64, i64, i32, i32, i32, f64, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz,
                            vp], i32),
        "cabs_kmeans_workspace_size": ([i64, i32, i32, i32, i32, P(sz)], i32),
        "cabs_kmeans": ([vp, vp, i64, i32, vp, i32, i32, i32, f32, vp, vp, vp, vp, vp, sz, vp], i32),
        "cabs_snap_workspace_size": ([i64, i32, i32, i32, P(sz)], i32),
        "cabs_snap": ([vp, vp, i64, i32, vp, i32, i32, vp, vp, vp, sz, vp], i32),
        "cabs_threshold_workspace_size": ([i64, P(sz)], i32),
        "cabs_threshold": ([vp, vp, i64, i32, i32, i32, vp, vp, sz, vp], i32),
        "cabs_orthogonalize_workspace_size": ([i64, i64, i32, i32, P(sz)], i32),
        "cabs_sketch_cur_workspace_size": ([P(cabs_source), P(cabs_cur_params), P(sz)], i32),
        "cabs_sketch_cur": ([vp, P(cabs_source), P(cabs_cur_params), vp, sz, vp, P(cabs_cur_result)], i32),
        "cabs_orthogonalize": ([vp, i64, i64, i32, i32, f64, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp], i32),
        "cabs_serve_start": ([vp, vp, sz, i32], i32),
        "cabs_serve_submit": ([vp, P(cabs_source), P(cabs_params), P(u64)], i32),
        "cabs_serve_poll": ([vp, u64, P(cabs_result), P(f64), i32], i32),
        "cabs_serve_release": ([vp, u64], i32),
        "cabs_serve_stop": ([vp], i32),
        "cabs_profile_enable": ([vp, i32], i32),
        "cabs_profile_read": ([vp, C.c_char_p, i32, P(i64), P(f64), i32, i32], i32),
        "cabs_launch_count": ([], i64),
        "cabs_error_noalloc": ([vp, P(cabs_source), P(cabs_params), P(cabs_result), i64, u64, vp, P(f64)], i32),
        "cabs_set_wait_limit": ([vp, i64], i32),
        "cabs_tune_set": ([vp, i32, i32, i64, i64, P(cabs_tune)], i32),
        "cabs_tune_get": ([vp, i32, i32, i64, i64, P(cabs_tune), P(i32)], i32),
        "cabs_tune_save": ([vp, C.c_char_p], i32),
        "cabs_tune_load": ([vp, C.c_char_p], i32),
        "cabs_autotune": ([vp, i32, P(cabs_source), P(cabs_params), vp, P(sz), P(cabs_result), vp, P(i32)], i32),
        "cabs_serve_times": ([vp, u64, P(f64), P(f64)], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def exported_names():
    return ["cabs_create", "cabs_destroy", "cabs_last_error", "cabs_version", "cabs_workspace_size", "cabs_sketch",
            "cabs_sketch_batched", "cabs_error_workspace_size", "cabs_error", "cabs_draw_indices", "cabs_gather",
            "cabs_sketching_workspace_size", "cabs_sketching", "cabs_kmeans_workspace_size", "cabs_kmeans",
            "cabs_snap_workspace_size", "cabs_snap", "cabs_threshold_workspace_size", "cabs_threshold",
            "cabs_orthogonalize_workspace_size", "cabs_orthogonalize", "cabs_sketch_cur_workspace_size",
            "cabs_sketch_cur", "cabs_serve_start", "cabs_serve_submit", "cabs_serve_poll",
            "cabs_serve_release", "cabs_serve_stop", "cabs_profile_enable", "cabs_profile_read",
            "cabs_launch_count", "cabs_error_noalloc", "cabs_set_wait_limit", "cabs_tune_set", "cabs_tune_get",
            "cabs_tune_save", "cabs_tune_load", "cabs_autotune", "cabs_serve_times"]


def _check(status, ctx=None):
    if status != CABS_OK:
        msg = lib().cabs_last_error(ctx)
        raise CabsError(status, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (row-major, as libcabs expects)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("libcabs takes row-major contiguous tensors; got strides %s" % (t.stride(),))
    if not t.is_cuda:
        raise ValueError("libcabs takes CUDA tensors")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ws(nbytes, device):
    import torch
    return torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=device)


def _aligned(ws):
    p = ws.data_ptr()
    return C.c_void_p((p + 255) & ~255), ws.numel() - ((-p) & 255)


# ------------------------------------------------------------------ context

class Context:
    """A libcabs context on one CUDA device."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().cabs_create(C.byref(h), device))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().cabs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cabs_version():
    return lib().cabs_version().decode()


WAIT_LIMIT_DEFAULT = 16777216


def cabs_set_wait_limit(ctx: Context, polls: int):
    """Polls before a grid-wide barrier gives up (kernels enqueued from now
    on); polls < 0 restores the default. A test control of the bounded waits."""
    _check(lib().cabs_set_wait_limit(ctx.h, int(polls)), ctx.h)


# ------------------------------------------------------------------ sources

@dataclass
class Source:
    """Keeps the tensors of a cabs_source alive."""
    c: cabs_source
    tensors: tuple


def dense_source(A, n=None):
    """A dense row-major FP32/FP64 CUDA matrix (may be a column slice of a wider one)."""
    import torch
    assert A.is_cuda and A.dim() == 2 and A.stride(1) == 1
    c = cabs_source(kind=SRC_DENSE, A=A.data_ptr(), lda=A.stride(0), a_is_f64=int(A.dtype == torch.float64))
    return Source(c, (A,))


def rbf_source(X, Y, sigma):
    """Implicit RBF kernel matrix from FP32 CUDA points X (m x d), Y (n x d)."""
    import torch
    assert X.is_cuda and Y.is_cuda and X.dtype == torch.float32 and Y.dtype == torch.float32
    X, Y = X.contiguous(), Y.contiguous()
    c = cabs_source(kind=SRC_RBF, X=X.data_ptr(), Y=Y.data_ptr(), d=X.shape[1], sigma=float(sigma))
    return Source(c, (X, Y))


def csr_source(row_ptr, col_idx, vals):
    """A sparse matrix in compressed rows on the device: row_ptr (m + 1, int64),
    col_idx (nnz, int32, sorted within rows), vals (nnz, FP32 or FP64)."""
    import torch
    assert row_ptr.is_cuda and row_ptr.dtype == torch.int64
    assert col_idx.is_cuda and col_idx.dtype == torch.int32 and vals.is_cuda
    row_ptr, col_idx, vals = row_ptr.contiguous(), col_idx.contiguous(), vals.contiguous()
    c = cabs_source(kind=SRC_CSR, A=vals.data_ptr(), a_is_f64=int(vals.dtype == torch.float64),
                    row_ptr=row_ptr.data_ptr(), col_idx=col_idx.data_ptr(), nnz=vals.numel())
    return Source(c, (row_ptr, col_idx, vals))


def make_params(m, n, k1, k2=None, iters=5, seed=1607, prec="fp64", core="pinv", upsilon_pow=0.0, trunc_rtol=0.0,
                flags=0, err_samples=None, err_seed=1607):
    """cabs_params; err_samples (0 = exact, > 0 = sampled) also sets CABS_FLAG_ERROR."""
    if err_samples is not None:
        flags |= FLAG_ERROR
    return cabs_params(m=m, n=n, k1=k1, k2=k1 if k2 is None else k2, iters=iters, seed=seed,
                       prec=PRECS[prec] if isinstance(prec, str) else prec,
                       core=CORES[core] if isinstance(core, str) else core, upsilon_pow=upsilon_pow,
                       trunc_rtol=trunc_rtol, flags=flags, err_samples=err_samples or 0, err_seed=err_seed)


def elem_dtype(prec):
    import torch
    p = PRECS[prec] if isinstance(prec, str) else prec
    return torch.float64 if p == PREC_FP64 else torch.float32


# ----------------------------------------------------------- whole sketch

@dataclass
class Sketch:
    U: object
    S: object
    V: object
    rows: object
    cols: object
    pilot_rows: object
    pilot_cols: object
    diag_buf: object
    params: cabs_params
    result: cabs_result = None
    err: object = None  # 1 FP64 device scalar: the relative error (CABS_FLAG_ERROR)

    def diag(self) -> cabs_diag:
        """Copies the device diagnostics to the host (synchronises)."""
        raw = bytes(self.diag_buf.cpu().numpy().tobytes())
        return cabs_diag.from_buffer_copy(raw[:C.sizeof(cabs_diag)])


def alloc_result(p: cabs_params, device="cuda"):
    import torch
    dt = elem_dtype(p.prec)
    U = torch.empty(p.m, p.k2, dtype=dt, device=device)
    S = torch.empty(p.k2, dtype=torch.float64, device=device)
    V = torch.empty(p.n, p.k2, dtype=dt, device=device)
    i32 = dict(dtype=torch.int32, device=device)
    rows, cols = torch.empty(p.k2, **i32), torch.empty(p.k2, **i32)
    prow, pcol = torch.empty(p.k1, **i32), torch.empty(p.k1, **i32)
    diag = torch.zeros(C.sizeof(cabs_diag), dtype=torch.uint8, device=device)
    err = torch.zeros(1, dtype=torch.float64, device=device)
    res = cabs_result(U=U.data_ptr(), S=S.data_ptr(), V=V.data_ptr(), rows=rows.data_ptr(), cols=cols.data_ptr(),
                      pilot_rows=prow.data_ptr(), pilot_cols=pcol.data_ptr(), diag=diag.data_ptr(),
                      err=err.data_ptr())
    return Sketch(U, S, V, rows, cols, prow, pcol, diag, p, res, err)


def cabs_workspace_size(src: Source, p: cabs_params) -> int:
    n = C.c_size_t()
    _check(lib().cabs_workspace_size(C.byref(src.c), C.byref(p), C.byref(n)))
    return n.value


def cabs_sketch(ctx: Context, src: Source, p: cabs_params, ws=None, out: Sketch = None, stream=None) -> Sketch:
    """One CABS sketch (Algorithm 2); outputs and workspace from torch."""
    import torch
    dev = torch.device("cuda", ctx.device)
    need = cabs_workspace_size(src, p)
    if ws is None or ws.numel() < need + 256:
        ws = _ws(need, dev)
    out = out or alloc_result(p, dev)
    wp, wn = _aligned(ws)
    _check(lib().cabs_sketch(ctx.h, C.byref(src.c), C.byref(p), wp, wn, _stream(stream), C.byref(out.result)),
           ctx.h)
    out._ws = ws
    return out


def cabs_sketch_batched(ctx: Context, srcs, params, outs, ws, offsets, lanes=4, use_graph=True, stream=None):
    n = len(srcs)
    SA = (cabs_source * n)(*[s.c for s in srcs])
    PA = (cabs_params * n)(*params)
    RA = (cabs_result * n)(*[o.result for o in outs])
    OA = (C.c_size_t * n)(*offsets)
    wp, _ = _aligned(ws)
    _check(lib().cabs_sketch_batched(ctx.h, n, SA, PA, wp, OA, RA, lanes, int(use_graph), _stream(stream)), ctx.h)


def cabs_tune_set(ctx: Context, p: cabs_params, tune=None):
    """Sets (tune: a cabs_tune or a dict of its fields) or removes (None) the
    launch shape of the bucket of p's (prec, k2, m, n)."""
    t = None
    if tune is not None:
        t = tune if isinstance(tune, cabs_tune) else cabs_tune(**tune)
    _check(lib().cabs_tune_set(ctx.h, p.prec, p.k2, p.m, p.n, C.byref(t) if t is not None else None), ctx.h)


def cabs_tune_get(ctx: Context, p: cabs_params):
    """(dict of the launch shape in force for p's bucket, found)."""
    t = cabs_tune()
    f = C.c_int32()
    _check(lib().cabs_tune_get(ctx.h, p.prec, p.k2, p.m, p.n, C.byref(t), C.byref(f)), ctx.h)
    return dict(extrap_tn=t.extrap_tn, gather_rows=t.gather_rows, assign_bn=t.assign_bn), bool(f.value)


def cabs_tune_save(ctx: Context, path: str):
    _check(lib().cabs_tune_save(ctx.h, path.encode()), ctx.h)


def cabs_tune_load(ctx: Context, path: str):
    _check(lib().cabs_tune_load(ctx.h, path.encode()), ctx.h)


def cabs_autotune(ctx: Context, srcs, params, outs, ws, offsets, stream=None) -> int:
    """Fills the context's launch-shape table from timed trials on the batch
    (whose outputs it overwrites) and returns the lanes it chose."""
    n = len(srcs)
    SA = (cabs_source * n)(*[s.c for s in srcs])
    PA = (cabs_params * n)(*params)
    RA = (cabs_result * n)(*[o.result for o in outs])
    OA = (C.c_size_t * n)(*offsets)
    wp, _ = _aligned(ws)
    lanes = C.c_int32()
    _check(lib().cabs_autotune(ctx.h, n, SA, PA, wp, OA, RA, _stream(stream), C.byref(lanes)), ctx.h)
    return lanes.value


def batched_layout(srcs, params):
    """Byte offsets (256-aligned) of each member's workspace slice and the total."""
    offs, tot = [], 0
    for s, p in zip(srcs, params):
        offs.append(tot)
        tot += (cabs_workspace_size(s, p) + 255) & ~255
    return offs, tot


def cabs_error(ctx: Context, src: Source, p: cabs_params, sk: Sketch, samples=0, seed=1607, stream=None) -> float:
    import torch
    nb = C.c_size_t()
    _check(lib().cabs_error_workspace_size(C.byref(src.c), C.byref(p), samples, C.byref(nb)))
    ws = _ws(nb.value, torch.device("cuda", ctx.device))
    wp, wn = _aligned(ws)
    out = C.c_double()
    _check(lib().cabs_error(ctx.h, C.byref(src.c), C.byref(p), C.byref(sk.result), samples, seed, wp, wn,
                            _stream(stream), C.byref(out)), ctx.h)
    return out.value


def cabs_error_noalloc(ctx: Context, src: Source, p: cabs_params, sk: Sketch, samples=0, seed=1607,
                       stream=None) -> float:
    """cabs_error for callers that cannot allocate device memory: no workspace,
    scratch in a fixed device array inside libcabs (exact error: m <= 1,048,576)."""
    out = C.c_double()
    _check(lib().cabs_error_noalloc(ctx.h, C.byref(src.c), C.byref(p), C.byref(sk.result), samples, seed,
                                    _stream(stream), C.byref(out)), ctx.h)
    return out.value


# ------------------------------------------------------------ step calls

def cabs_draw_indices(ctx: Context, seed, tag, N, k, stream=None):
    import torch
    dev = torch.device("cuda", ctx.device)
    drawn = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
    srt = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
    _check(lib().cabs_draw_indices(ctx.h, seed, tag, N, k, _ptr(drawn), _ptr(srt), _stream(stream)), ctx.h)
    return drawn[:k], srt[:k]


def cabs_gather(ctx: Context, src: Source, m, n, rows, cols, prec="fp64", want=("C", "Rt", "W"), stream=None):
    import torch
    dev = torch.device("cuda", ctx.device)
    dt = elem_dtype(prec)
    kr, kc = rows.numel(), cols.numel()
    Cm = torch.empty(m, kc, dtype=dt, device=dev) if "C" in want else None
    Rt = torch.empty(n, kr, dtype=dt, device=dev) if "Rt" in want else None
    W = torch.empty(kr, kc, dtype=torch.float64, device=dev) if "W" in want else None
    p = PRECS[prec] if isinstance(prec, str) else prec
    _check(lib().cabs_gather(ctx.h, C.byref(src.c), m, n, _ptr(rows), kr, _ptr(cols), kc, p, _ptr(Cm), _ptr(Rt),
                             _ptr(W), _stream(stream)), ctx.h)
    return Cm, Rt, W


def cabs_sketching(ctx: Context, Cm, Rt, W, m, n, prec="fp64", core="pinv", trunc_rtol=0.0, embed=False,
                   stream=None):
    import torch
    dev = torch.device("cuda", ctx.device)
    k = W.shape[0]
    p = PRECS[prec] if isinstance(prec, str) else prec
    dt = elem_dtype(p)
    nb = C.c_size_t()
    _check(lib().cabs_sketching_workspace_size(m, n, k, p, C.byref(nb)))
    ws = _ws(nb.value, dev)
    wp, wn = _aligned(ws)
    out1 = torch.empty(m, k, dtype=dt, device=dev)
    out2 = torch.empty(n, k, dtype=dt, device=dev)
    S = torch.empty(k, dtype=torch.float64, device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    rank, sweeps = torch.zeros(1, **i32), torch.zeros(1, **i32)
    sig = torch.empty(k, dtype=torch.float64, device=dev)
    Uw = torch.empty(k, k, dtype=torch.float64, device=dev)
    Vw = torch.empty(k, k, dtype=torch.float64, device=dev)
    c = CORES[core] if isinstance(core, str) else core
    _check(lib().cabs_sketching(ctx.h, m, n, k, p, c, trunc_rtol, _ptr(Cm), _ptr(Rt), _ptr(W), int(embed), _ptr(out1),
                                _ptr(S), _ptr(out2), _ptr(rank), _ptr(sweeps), _ptr(sig), _ptr(Uw), _ptr(Vw), wp, wn,
                                _stream(stream)), ctx.h)
    return dict(out1=out1, S=S, out2=out2, rank=rank, sweeps=sweeps, sig=sig, Uw=Uw, Vw=Vw, ws=ws)


def cabs_kmeans(ctx: Context, X, init_rows, k2, iters, prec="fp64", upsilon_pow=0.0, stream=None):
    import torch
    dev = torch.device("cuda", ctx.device)
    M, d = X.shape
    p = PRECS[prec] if isinstance(prec, str) else prec
    nb = C.c_size_t()
    _check(lib().cabs_kmeans_workspace_size(M, d, k2, iters, p, C.byref(nb)))
    ws = _ws(nb.value, dev)
    wp, wn = _aligned(ws)
    labels = torch.empty(max(iters, 1), M, dtype=torch.int32, device=dev)
    centres = torch.empty(k2, d, dtype=X.dtype, device=dev)
    energy = torch.zeros(max(iters, 1), dtype=torch.float64, device=dev)
    T = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib().cabs_kmeans(ctx.h, _ptr(X), M, d, _ptr(init_rows), k2, iters, p, upsilon_pow, _ptr(labels),
                             _ptr(centres), _ptr(energy), _ptr(T), wp, wn, _stream(stream)), ctx.h)
    return dict(labels=labels[:iters], centres=centres, energy=energy[:iters], T=T, ws=ws)


def cabs_snap(ctx: Context, X, Z, prec="fp64", stream=None):
    import torch
    dev = torch.device("cuda", ctx.device)
    M, d = X.shape
    k2 = Z.shape[0]
    p = PRECS[prec] if isinstance(prec, str) else prec
    nb = C.c_size_t()
    _check(lib().cabs_snap_workspace_size(M, d, k2, p, C.byref(nb)))
    ws = _ws(nb.value, dev)
    wp, wn = _aligned(ws)
    order = torch.empty(k2, dtype=torch.int32, device=dev)
    srt = torch.empty(k2, dtype=torch.int32, device=dev)
    _check(lib().cabs_snap(ctx.h, _ptr(X), M, d, _ptr(Z), k2, p, _ptr(order), _ptr(srt), wp, wn, _stream(stream)),
           ctx.h)
    return order, srt


def cabs_threshold(ctx: Context, X, k2, prec="fp64", stream=None):
    """Section 5 follow-up variant (f): the k2 largest-norm rows of X, sorted (device int32)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    M, d = X.shape
    p = PRECS[prec] if isinstance(prec, str) else prec
    nb = C.c_size_t()
    _check(lib().cabs_threshold_workspace_size(M, C.byref(nb)))
    ws = _ws(nb.value, dev)
    wp, wn = _aligned(ws)
    srt = torch.empty(k2, dtype=torch.int32, device=dev)
    _check(lib().cabs_threshold(ctx.h, _ptr(X), M, d, k2, p, _ptr(srt), wp, wn, _stream(stream)), ctx.h)
    return srt


def cabs_orthogonalize(ctx: Context, U, S, V, prec="fp64", trunc_rtol=0.0, stream=None):
    """Supplementary Section 3: U diag(S) V^T -> X diag(s) Y^T with orthonormal X, Y.
    Returns (X, s, Y, rank) on the device; columns and s beyond rank are zero."""
    import torch
    dev = torch.device("cuda", ctx.device)
    m, k = U.shape
    n = V.shape[0]
    p = PRECS[prec] if isinstance(prec, str) else prec
    nb = C.c_size_t()
    _check(lib().cabs_orthogonalize_workspace_size(m, n, k, p, C.byref(nb)))
    ws = _ws(nb.value, dev)
    wp, wn = _aligned(ws)
    X = torch.empty(m, k, dtype=U.dtype, device=dev)
    Y = torch.empty(n, k, dtype=V.dtype, device=dev)
    s = torch.empty(k, dtype=torch.float64, device=dev)
    rank = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib().cabs_orthogonalize(ctx.h, m, n, k, p, trunc_rtol, _ptr(U), _ptr(S), _ptr(V), _ptr(X), _ptr(s),
                                    _ptr(Y), _ptr(rank), wp, wn, _stream(stream)), ctx.h)
    return X, s, Y, rank


class CurSketch:
    """Device outputs of one Sketch-CUR: A ~ U diag(S) V^T with U = C U*, S = 1, V = R^T."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def make_cur_params(m, n, kb, kt=None, seed=1607, prec="fp64", trunc_rtol=0.0):
    p = PRECS[prec] if isinstance(prec, str) else prec
    return cabs_cur_params(m=m, n=n, kb=kb, kt=3 * kb if kt is None else kt, seed=seed, prec=p,
                           trunc_rtol=trunc_rtol)


def cabs_sketch_cur(ctx: Context, src: Source, p: cabs_cur_params, stream=None, ws=None):
    """Section 2.2, Algorithm 1 as Sketch-CUR (see cabs.h)."""
    import torch
    dev = torch.device("cuda", ctx.device)
    nb = C.c_size_t()
    _check(lib().cabs_sketch_cur_workspace_size(C.byref(src.c), C.byref(p), C.byref(nb)))
    if ws is None or ws.numel() < nb.value + 256:
        ws = _ws(nb.value, dev)
    wp, wn = _aligned(ws)
    dt = elem_dtype(p.prec)
    i32 = dict(dtype=torch.int32, device=dev)
    o = CurSketch(U=torch.empty(p.m, p.kb, dtype=dt, device=dev), S=torch.empty(p.kb, dtype=torch.float64, device=dev),
                  V=torch.empty(p.n, p.kb, dtype=dt, device=dev),
                  Ustar=torch.empty(p.kb, p.kb, dtype=torch.float64, device=dev),
                  rows_b=torch.empty(p.kb, **i32), cols_b=torch.empty(p.kb, **i32),
                  rows_t=torch.empty(p.kt, **i32), cols_t=torch.empty(p.kt, **i32), ranks=torch.zeros(8, **i32),
                  ws=ws)
    res = cabs_cur_result(U=_ptr(o.U), S=_ptr(o.S), V=_ptr(o.V), Ustar=_ptr(o.Ustar), rows_b=_ptr(o.rows_b),
                          cols_b=_ptr(o.cols_b), rows_t=_ptr(o.rows_t), cols_t=_ptr(o.cols_t), ranks=_ptr(o.ranks))
    _check(lib().cabs_sketch_cur(ctx.h, C.byref(src.c), C.byref(p), wp, wn, _stream(stream), C.byref(res)), ctx.h)
    # the factor form U diag(S) V^T, as cabs_error takes it
    o.result = cabs_result(U=_ptr(o.U), S=_ptr(o.S), V=_ptr(o.V), rows=_ptr(o.rows_b), cols=_ptr(o.cols_b),
                           pilot_rows=_ptr(o.rows_b), pilot_cols=_ptr(o.cols_b), diag=None, err=None)
    return o


# -------------------------------------------------------------- profiling

def cabs_profile_enable(ctx: Context, on: bool = True):
    _check(lib().cabs_profile_enable(ctx.h, int(on)), ctx.h)


def cabs_profile_read(ctx: Context, reset: bool = True, max_rows: int = 128):
    """{kernel name: (launches, total device ms)} since the last reset."""
    name_len = 64
    names = C.create_string_buffer(max_rows * name_len)
    launches = (C.c_int64 * max_rows)()
    ms = (C.c_double * max_rows)()
    n = lib().cabs_profile_read(ctx.h, names, name_len, launches, ms, max_rows, int(reset))
    out = {}
    for i in range(n):
        nm = names.raw[i * name_len:(i + 1) * name_len].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


def cabs_launch_count() -> int:
    return int(lib().cabs_launch_count())


# ---------------------------------------------------------------- serving

class Server:
    """cabs_serve_* over a torch-allocated HBM arena."""

    def __init__(self, ctx: Context, arena_bytes: int, max_slots: int = 8):
        import torch
        self.ctx = ctx
        self.arena = torch.empty(arena_bytes + 256, dtype=torch.uint8, device=torch.device("cuda", ctx.device))
        wp, wn = _aligned(self.arena)
        _check(lib().cabs_serve_start(ctx.h, wp, wn, max_slots), ctx.h)
        self.sources = {}

    def submit(self, src: Source, p: cabs_params) -> int:
        t = C.c_uint64()
        _check(lib().cabs_serve_submit(self.ctx.h, C.byref(src.c), C.byref(p), C.byref(t)), self.ctx.h)
        self.sources[t.value] = (src, p)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """Returns (cabs_result, latency_ms), or None while the request is not finished."""
        res = cabs_result()
        lat = C.c_double()
        st = lib().cabs_serve_poll(self.ctx.h, ticket, C.byref(res), C.byref(lat), timeout_ms)
        if st == CABS_EBUSY:
            return None
        _check(st, self.ctx.h)
        return res, lat.value

    def times(self, ticket: int):
        """(start_ms, end_ms): the finished request's device-side interval since the loop started."""
        a, b = C.c_double(), C.c_double()
        _check(lib().cabs_serve_times(self.ctx.h, ticket, C.byref(a), C.byref(b)), self.ctx.h)
        return a.value, b.value

    def release(self, ticket: int):
        _check(lib().cabs_serve_release(self.ctx.h, ticket), self.ctx.h)
        self.sources.pop(ticket, None)

    def stop(self):
        _check(lib().cabs_serve_stop(self.ctx.h), self.ctx.h)


class _DevView:
    """A device buffer described by __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = dict(shape=tuple(shape), typestr=typestr, data=(int(ptr), False),
                                             version=3, strides=None)


def result_err(res: cabs_result, device="cuda") -> float:
    """The relative error a request computed with CABS_FLAG_ERROR (reads one
    FP64 device scalar of the serving arena)."""
    import torch
    if not res.err:
        raise ValueError("the result carries no error (CABS_FLAG_ERROR was not set)")
    return float(torch.as_tensor(_DevView(res.err, (1,), "<f8"), device=device).cpu()[0])


def result_tensors(res: cabs_result, p: cabs_params, device="cuda"):
    """Copies a serving result (device pointers into the arena) into new torch tensors."""
    import torch
    f = "<f8" if p.prec == PREC_FP64 else "<f4"

    def grab(ptr, shape, ts):
        return torch.as_tensor(_DevView(ptr, shape, ts), device=device).clone()

    U = grab(res.U, (p.m, p.k2), f)
    S = grab(res.S, (p.k2,), "<f8")
    V = grab(res.V, (p.n, p.k2), f)
    rows = grab(res.rows, (p.k2,), "<i4")
    cols = grab(res.cols, (p.k2,), "<i4")
    return U, S, V, rows, cols
