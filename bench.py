"""Benchmark of the CABS hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cabs|reference]
                    [--workload dense|rbf|plain] [--prec bf16|tf32|fp32|fp64]
                    [--form batched|plain] [--batch B] [--lanes L]

One sketch is one pass of the whole hot path over one synthetic input: pilot
draw, gathers, FP64 core, embeddings, weighted k-means on both sides, snap,
follow-up gather and core (Algorithm 2), then the relative Frobenius error
(exact for dense inputs, 10^6 sampled entries for the implicit RBF matrix).

A step is B independent sketches of the same matrix (seeds differ) and their
errors. The default (batched) form enqueues them over L streams as one
captured CUDA graph, so that one sketch's narrow phases (the core SVD runs on
one thread-block cluster) overlap another's bandwidth-bound ones; --form plain
runs one sketch per step. The same line also carries the plain FP32 form (one
sketch at a time, no graph) for comparison.

Inputs are resident in HBM before the timed region; the dense workload's A
(8 GiB) is larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank sketches its
own matrix (replicas; no collective on the data path) and `value` counts the
sketches of all ranks over the slowest rank's time.

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload (see cpu_sample()).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CABS sketches/s and p50/p99 latency at stated rel. Frobenius error; gather GB/s"

# Truncation of W's spectrum (Section 4.1 leaves it open): singular values
# below k u sigma_1 are not resolved by the data when its entries carry the unit
# roundoff u, so the FP32 workloads (stored FP32 A, RBF entries generated in
# FP32) keep sigma_i > k 2^-24 sigma_1 and the FP64 one k 2^-52 (the library's
# default). For the pseudo-inverse core this is what keeps noise directions
# of W from being amplified by 1 / sigma_i.
U_FP32 = 2.0 ** -24


def trunc_rtol(wl, k):
    return k * U_FP32 if wl["kind"] in ("dense", "rbf", "csr") else 0.0


WORKLOADS = {
    # dense stored FP32 A, 65536 x 32768 (8 GiB): the headline workload
    "dense": dict(kind="dense", m=65536, n=32768, rank=256, k=256, iters=5, core="stabilized",
                  desc="dense FP32 A 65536x32768 = U diag(exp(-i/30)) V^T (rank 256) + N(0,1e-4^2); k=256, c=5"),
    # implicit RBF matrix, 1e5 x 1e5 points in d=16
    "rbf": dict(kind="rbf", m=100000, n=100000, d=16, k=200, iters=10, core="pinv", samples=1000000,
                desc="implicit RBF exp(-|x-y|^2/2s^2), 1e5 x 1e5 points d=16 (50-comp. mixture); k=200, c=10"),
    # plain FP64 2000 x 1500 (the small case the oracle finishes in seconds)
    "plain": dict(kind="plain", m=2000, n=1500, k=20, iters=5, core="pinv",
                  desc="plain FP64 A 2000x1500 = U V^T + N(0,1e-6); k=20, c=5"),
    # Table 1's movie-ratings shape: sparse CSR
    "sparse": dict(kind="csr", m=27000, n=46000, density=0.0056, k=256, iters=5, core="stabilized",
                   desc="sparse CSR A 27000x46000, 0.56 % (ratings-like, power-law rows and columns, rank-20 "
                        "values); k=256, c=5, exact error by the linear-cost identity"),
}

# Peaks: measured copy bandwidth and BF16 GEMM from MEASURED_PEAKS.json; the
# FP32, TF32 and FP64 peaks are measured at start-up the same way (a timed
# cuBLAS GEMM through torch, see measure_alu_peaks). The unit-count figures
# (152 SMs x 128 FP32 lanes or 2 FP64 lanes x 2 flops x 2.07 GHz) are
# reported beside them, and used only when the measurement fails.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measure_alu_peaks(device):
    """FP32 (no TF32), TF32 and FP64 GEMM throughput of this GPU: torch.matmul
    of n x n operands (n = 8192 FP32/TF32, 4096 FP64), 2 n^3 flops, fastest of
    5 after 2 warm-up products, CUDA events on the current stream."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, tf32, n in (("fp32", torch.float32, False, 8192), ("tf32", torch.float32, True, 8192),
                                  ("fp64", torch.float64, False, 4096)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            g = torch.Generator(device=device)
            g.manual_seed(5)
            a = torch.randn(n, n, device=device, dtype=dt, generator=g)
            b = torch.randn(n, n, device=device, dtype=dt, generator=g)
            for _ in range(2):
                torch.matmul(a, b)
            best = float("inf")
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            out[name + "_tflops"] = round(2.0 * n ** 3 / best / 1e12, 2)
            del a, b
    except Exception as e:  # noqa: BLE001 -- the derived figures stand in
        out["error"] = str(e)[:200]
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), bf16_tflops=float(p["bf16_tflops"]),
                    bf16_tflops_sustained=float(p["bf16_tflops_sustained"]), source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, source="fallback")


# ------------------------------------------------------------------ inputs

def make_inputs(wl, device, seed=1607):
    import numpy as np
    import torch

    from workloads import synth
    if wl["kind"] == "dense":
        A, U, sv, V = synth.decaying_lowrank_device(wl["m"], wl["n"], rank=wl["rank"], seed=seed, device=device)
        return dict(A=A, L=(U, sv, V))
    if wl["kind"] == "rbf":
        X, Y, sig = synth.rbf_mixture(wl["m"], wl["n"], d=wl["d"], seed=seed)
        return dict(X=torch.from_numpy(X).to(device), Y=torch.from_numpy(Y).to(device), sigma=float(sig),
                    X_host=X, Y_host=Y)
    if wl["kind"] == "csr":
        ip, ix, v = synth.sparse_lowrank(wl["m"], wl["n"], wl["density"], seed=seed)
        return dict(row_ptr=torch.from_numpy(ip).to(device), col_idx=torch.from_numpy(ix).to(device),
                    vals=torch.from_numpy(v).to(device), host=(ip, ix, v))
    A = synth.plain_lowrank(wl["m"], wl["n"], seed=seed)
    return dict(A=torch.from_numpy(np.ascontiguousarray(A)).to(device))


def noiseless_error(L, sk):
    """|L - U_bar S_bar V_bar^T|_F / |L|_F against the noiseless part L = U_L diag(s) V_L^T
    of the dense input, by k x k algebra in FP64 (U_L, V_L orthonormal):
    <L, X> = sum_ab s_a (U_L^T U_bar)_ab S_b (V_L^T V_bar)_ab,
    |X|^2 = sum_bc S_b S_c (U_bar^T U_bar)_bc (V_bar^T V_bar)_bc. A diagnostic outside
    the timed region (torch arithmetic, not the product path)."""
    import torch
    UL, s, VL = L
    U, S, V = sk.U.double(), sk.S.double(), sk.V.double()
    M1, M2 = UL.T @ U, VL.T @ V
    lx = ((s[:, None] * M1) * (M2 * S[None, :])).sum()
    xx = (S[:, None] * (U.T @ U) * S[None, :] * (V.T @ V)).sum()
    ll = (s * s).sum()
    return float(torch.sqrt(torch.clamp(ll - 2 * lx + xx, min=0.0) / ll))


def precision_excess(cabs, ctx, wl, device):
    """Relative error of each precision mode on the oracle-sized slice of the
    workload (same recipe and seed as the CPU baseline's first oracle step), and
    its relative excess over the FP64 mode (which matches the oracle to 1e-10)."""
    import numpy as np
    import torch

    from workloads import synth
    s = cpu_sample(wl)
    if wl["kind"] == "dense":
        A = synth.decaying_lowrank_host(s["m"], s["n"], rank=wl["rank"], seed=1607)[0]
        src = cabs.dense_source(torch.from_numpy(A).to(device))
        samples = 0
    elif wl["kind"] == "csr":
        ip, ix, v = synth.sparse_lowrank(s["m"], s["n"], wl["density"], seed=1607)
        src = cabs.csr_source(torch.from_numpy(ip).to(device), torch.from_numpy(ix).to(device),
                              torch.from_numpy(v).to(device))
        samples = 0
    else:
        X, Y, sig = synth.rbf_mixture(s["m"], s["n"], d=wl["d"], seed=1607)
        src = cabs.rbf_source(torch.from_numpy(X).to(device), torch.from_numpy(Y).to(device), sig)
        samples = s["samples"]
    errs, unsupported = {}, {}
    for prec in ("fp64", "fp32", "tf32", "bf16"):
        p = cabs.make_params(s["m"], s["n"], s["k"], iters=s["iters"], seed=1607, prec=prec, core=wl["core"],
                             trunc_rtol=trunc_rtol(wl, s["k"]),
                             err_samples=samples, err_seed=3)
        try:
            sk = cabs.cabs_sketch(ctx, src, p)
        except cabs.CabsError as e:  # e.g. TF32 k-means beyond its embedding width
            unsupported[prec] = str(e)
            continue
        errs[prec] = float(sk.err.cpu().item())
    torch.cuda.synchronize()
    return dict(slice=f"{s['m']}x{s['n']}, k={s['k']}, c={s['iters']}, seed 1607", errors=errs,
                excess_over_fp64={p_: errs[p_] / errs["fp64"] - 1.0 for p_ in ("fp32", "tf32", "bf16") if p_ in errs},
                unsupported=unsupported or None, bar=1e-3)


def make_source(cabs, wl, inp):
    if wl["kind"] == "rbf":
        return cabs.rbf_source(inp["X"], inp["Y"], inp["sigma"])
    if wl["kind"] == "csr":
        return cabs.csr_source(inp["row_ptr"], inp["col_idx"], inp["vals"])
    return cabs.dense_source(inp["A"])


# ------------------------------------------------------- algorithmic units

def algorithmic(name, wl, k, iters, elem_bytes, svd_sweeps, svd_refine=None):
    """(bound, algorithmic amount per step, unit, launches per step) of a kernel.

    Per-unit figures: gathers read one 32-byte DRAM sector per scattered
    element of C plus the coalesced row reads, and write C and Rt; the exact
    residual reads A once (m n 4 bytes); contractions count 2 flops per
    multiply-add (k-means: 2 (m + n) k^2 per iteration; extrapolation
    2 (m + n) k^2 per round; snap candidates 3 (m + n) k^2); the FP32 Jacobi
    sweep counts 18 k flops per column pair."""
    m, n = wl["m"], wl["n"]
    d = k
    kp = (k + 63) // 64 * 64
    if name == "residual_dense_kernel":
        return "alu", 2.0 * m * n * k, "TFLOP/s", 1
    if name == "tc_residual_kernel":
        return "hbm", float(m) * n * 4, "GB/s", 1
    if name == "gather_cols_kernel":
        return "hbm", 2 * m * k * (32 + elem_bytes), "GB/s", 2
    if name == "gather_rows_t_kernel":
        return "hbm", 2 * 2 * n * k * elem_bytes, "GB/s", 2
    if name in ("svd32_cluster_kernel", "svd32_cta_kernel"):
        fl = sum(s * (k * (k - 1) / 2) * 18.0 * k for s in svd_sweeps)
        return "alu", fl, "TFLOP/s", 2
    if name == "svd_jacobi_kernel":
        fl = sum(s * (k * (k - 1) / 2) * 18.0 * k for s in svd_sweeps)
        return "alu", fl, "TFLOP/s", 2
    if name in ("assign_f32_kernel", "assign_f64_kernel"):
        return "alu", iters * 2.0 * (m + n) * k * d, "TFLOP/s", 2 * iters
    if name == "tc_assign_kernel":
        return "tensor", iters * 2.0 * (m + n) * k * kp, "TFLOP/s", 2 * iters
    if name == "tc_snap_kernel":
        return "tensor", 2.0 * (m + n) * k * kp, "TFLOP/s", 2
    if name == "refine_persistent_kernel":
        # iterations x (W V, U^T P, U^T U, V^T V, U F, V G): 6 k^3 multiply-adds, FP64
        its = sum(max(r, 0) for r in (svd_refine or (3, 3)))
        return "alu", its * 6 * 2.0 * k ** 3, "TFLOP/s", 2
    if name == "snap_cand_kernel":
        return "alu", 3.0 * (m + n) * k * d, "TFLOP/s", 2
    if name in ("extrap_gemm_kernel(X = U T_u)", "extrap_gemm_kernel(Y = V T_v)"):
        # the orthogonalisation's tall products (supplementary Section 3), once per sketch
        side = m if "X = U" in name else n
        return "alu", 2.0 * side * k * k, "TFLOP/s", 1
    if name.startswith("extrap_gemm_kernel"):
        side = m if "C V_w" in name else n
        return "alu", 2 * 2.0 * side * k * k, "TFLOP/s", 2
    if name == "gram_kernel":
        # U^T U and V^T V by upper-triangle tiles of 128 x 128 (FP32): two launches per sketch
        nt = (k + 127) // 128
        return "alu", 2.0 * (m + n) * (nt * (nt + 1) // 2) * 128 * 128, "TFLOP/s", 2
    if name == "lev_keys_kernel":
        # reads the orthonormal pilot factors once, writes one 8-byte key per row
        return "hbm", (m + n) * (k * elem_bytes + 8.0), "GB/s", 2
    if name in ("rbf_block_kernel(C)", "rbf_block_kernel(Rt)"):
        side = m if name.endswith("(C)") else n
        return "alu", 2 * side * k * (3.0 * wl.get("d", 16) + 20), "TFLOP/s", 2
    if name == "update_kernel":
        return "hbm", iters * (m + n) * d * elem_bytes, "GB/s", 2 * iters
    return None


def kernel_traffic(name, workload):
    """DRAM bytes per launch of a kernel from the committed ncu summary
    (profiles/ncu_traffic.json), or None when there is none for this workload
    or the kernel's source file has changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return None
    e = table.get(workload, {}).get(name)
    if not e:
        return None
    try:
        with open(os.path.join(ROOT, e["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != e["source_sha256"]:
                return None
    except OSError:
        return None
    return dict(bytes=int(e["dram_bytes_per_launch"]), captured_on=e["captured_on"], scaled=e.get("scaled"))


def roofline_of(name, launches, ms, wl, k, iters, elem_bytes, svd_sweeps, steps, peaks, prec, workload,
                svd_refine=None):
    info = algorithmic(name, wl, k, iters, elem_bytes, svd_sweeps, svd_refine)
    if info is None:
        return dict(kernel=name, bound=None, achieved=None, peak=None, unit=None, frac=None, traffic=None)
    bound, amount, unit, _ = info
    secs = ms / 1e3
    achieved = amount * steps / secs / (1e12 if unit == "TFLOP/s" else 1e9)
    if bound == "hbm":
        peak, src = peaks["hbm_gbs"], peaks["source"] + " copy"
    elif bound == "tensor":
        if prec == "bf16" or "tf32_tflops" not in peaks:
            peak = peaks["bf16_tflops_sustained"] if prec == "bf16" else peaks["bf16_tflops_sustained"] / 2
            src = peaks["source"] + (" bf16 sustained" if prec == "bf16" else " bf16 sustained / 2 (tf32 nominal ratio)")
        else:
            peak, src = peaks["tf32_tflops"], "measured cuBLAS TF32 GEMM 8192^3 (torch.matmul, start-up)"
    else:
        fp64 = name in ("svd_jacobi_kernel", "refine_persistent_kernel") or (prec == "fp64" and not name.startswith("svd32"))
        key = "fp64_tflops" if fp64 else "fp32_tflops"
        if key in peaks:
            peak = peaks[key]
            src = (f"measured cuBLAS {'D' if fp64 else 'S'}GEMM {'4096' if fp64 else '8192'}^3 (torch.matmul, "
                   f"start-up); unit-count figure {FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS:.2f}")
        else:
            peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
            src = "derived from unit counts x 2.07 GHz"
    tr = kernel_traffic(name, workload)
    extra = {}
    if name.startswith("svd32_cluster"):
        # one 16-CTA cluster: the fraction of the peak of the SMs it occupies
        extra = dict(sms_used=16, frac_of_sms_used=round(achieved / (peak * 16 / 152), 5))
    return dict(kernel=name, bound=bound, achieved=round(achieved, 4), peak=round(peak, 3), unit=unit, **extra,
                frac=round(achieved / peak, 5), traffic=tr["bytes"] if tr else None, peak_source=src,
                avg_launch_ms=round(ms / max(launches, 1), 5),
                traffic_source=(f"ncu capture ({tr['captured_on']})" + (f", {tr['scaled']}" if tr.get("scaled") else ""))
                if tr else None)


def roofline(prof, wl, k, iters, elem_bytes, svd_sweeps, steps, peaks, prec, workload, svd_refine=None):
    """Roofline of the kernel with the largest device time in the timed region
    (and of the next ones, for context), plus the per-kernel time table."""
    if not prof:
        return None, None, None
    total = sum(x[1] for x in prof.values())
    order = sorted(prof.items(), key=lambda kv: -kv[1][1])
    table = {nm: dict(launches=l, total_ms=round(t, 4), share=round(t / total, 4)) for nm, (l, t) in order}
    rl = [roofline_of(nm, l, t, wl, k, iters, elem_bytes, svd_sweeps, steps, peaks, prec, workload, svd_refine)
          for nm, (l, t) in order[:6]]
    return rl[0], table, rl[1:]


# ------------------------------------------------------------------ clocks

def bind_to_gpu_local_cpus(local):
    """Restricts this process to the CPUs that the GPU's PCI device lists as
    local (sysfs local_cpulist), so that pinned host buffers allocated after
    this land on the GPU's own memory node (first touch). Returns the list
    as a string, or why it was left unbound."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(local), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/local_cpulist"
        with open(path) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return "unbound (no local CPU available to this process)"
        os.sched_setaffinity(0, cpus)
        return spec
    except Exception as e:  # noqa: BLE001 -- the measurement runs unbound
        return f"unbound ({type(e).__name__})"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the first sample marks the sampler as running; the timed region starts after it
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        self.lines_before = sum(1 for _ in open(self.path))

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for i, ln in enumerate(open(self.path)):
            if i < getattr(self, "lines_before", 0):
                continue
            p = [x.strip() for x in ln.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows))


# -------------------------------------------------------------- CPU oracle

CPU_BUDGET_S = 90.0  # wall-clock cap on the oracle repeats of one baseline


def cpu_sample(wl):
    """The bounded oracle sample of a workload and how to scale its time.

    dense: the same recipe at 4096 x 2048 (k = 256, c = 5), the slice size the
           oracle comparison uses; sketch time scales with m + n, the exact
           error with m n.
    rbf:   the same recipe at 10^4 x 10^4 points (k = 200, c = 10), error on
           10^5 sampled entries; sketch time scales with m + n, the sampled
           error with the sample count.
    plain: the whole workload (no scaling)."""
    if wl["kind"] == "dense":
        return dict(m=4096, n=2048, k=wl["k"], iters=wl["iters"], scale_sketch=(wl["m"] + wl["n"]) / (4096 + 2048),
                    scale_err=(wl["m"] * wl["n"]) / (4096 * 2048))
    if wl["kind"] == "rbf":
        return dict(m=10000, n=10000, k=wl["k"], iters=wl["iters"], samples=100000,
                    scale_sketch=(wl["m"] + wl["n"]) / 20000, scale_err=wl["samples"] / 100000)
    if wl["kind"] == "csr":
        # one tenth of each side at the same density; the oracle's error is the
        # dense definition on the slice, scaled by m n
        return dict(m=wl["m"] // 10, n=wl["n"] // 10, k=wl["k"], iters=wl["iters"],
                    scale_sketch=10.0, scale_err=100.0)
    return dict(m=wl["m"], n=wl["n"], k=wl["k"], iters=wl["iters"], scale_sketch=1.0, scale_err=1.0)


def cpu_worker(workload, steps):
    """Runs in a child process with one BLAS thread: times the oracle."""
    import numpy as np

    from oracle import cabs_ref as o
    from workloads import synth
    wl = WORKLOADS[workload]
    s = cpu_sample(wl)
    if wl["kind"] == "dense":
        A = synth.decaying_lowrank_host(s["m"], s["n"], rank=wl["rank"], seed=1607)[0]
        src = o.DenseSource(A)
    elif wl["kind"] == "rbf":
        X, Y, sig = synth.rbf_mixture(s["m"], s["n"], d=wl["d"], seed=1607)
        src = o.RBFSource(X, Y, sig)
    elif wl["kind"] == "csr":
        ip, ix, v = synth.sparse_lowrank(s["m"], s["n"], wl["density"], seed=1607)
        src = o.CSRSource(ip, ix, v, s["n"])
        src.A_dense = src.dense()
    else:
        A = synth.plain_lowrank(s["m"], s["n"], seed=1607)
        src = o.DenseSource(A)
    times = []
    start = time.perf_counter()
    for step in range(steps):
        if step > 0 and time.perf_counter() - start > CPU_BUDGET_S:
            break  # bounded: the remaining repeats would not change the median much
        t0 = time.perf_counter()
        r = o.cabs(src, s["k"], iters=s["iters"], seed=1607 + step, mode=wl["core"], trunc_rtol=trunc_rtol(wl, s["k"]))
        t1 = time.perf_counter()
        if wl["kind"] == "rbf":
            err = o.rel_fro_error_sampled(src, r.final.U, r.final.S, r.final.V, 3, s["samples"])
        elif wl["kind"] == "csr":
            err = o.rel_fro_error_dense(src.A_dense, r.final.U, r.final.S, r.final.V)
        else:
            err = o.rel_fro_error_dense(src.A, r.final.U, r.final.S, r.final.V)
        t2 = time.perf_counter()
        times.append((t1 - t0) * s["scale_sketch"] + (t2 - t1) * s["scale_err"])
        if step == 0:
            err0 = err
    print(json.dumps(dict(times=times, err=err, err0=err0, sample=s)))


def run_cpu_baseline(workload, steps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", workload,
                          "--steps", str(steps)], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle worker failed:\n" + out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    s = res["sample"]
    per = statistics.median(res["times"])
    desc = (f"oracle on the same recipe at {s['m']}x{s['n']}, k={s['k']}, c={s['iters']}; sketch time x"
            f"{s['scale_sketch']:.3g} (m+n), error time x{s['scale_err']:.3g}; median of {len(res['times'])}")
    return dict(value=1.0 / per, unit="sketches/s", cores=1, kind="oracle", sample=desc,
                seconds_per_sketch_extrapolated=per, oracle_error=res.get("err0"))


# --------------------------------------------------------------- GPU arm

def rank_max(x, device=None):
    """Maximum of x over the ranks of the default process group (x alone
    without one): the slowest rank's time decides a whole-job number."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, sketches_per_rank_step, steps, total_ms):
    """Whole-job throughput: every rank's sketches over the slowest rank's time."""
    return world * sketches_per_rank_step * steps / (total_ms / 1e3)


def timed_steps(ctx, cabs, step, steps, stream, world, barrier, flush=None):
    """Runs `steps` steps between barriers; returns (per-step ms, total ms max over ranks, errors).

    With `flush` (inputs smaller than L2), each step is bracketed by its own
    event pair and flush() -- a write of a buffer larger than L2 -- runs
    between steps, outside the timed pairs; the total is the sum of the steps."""
    import torch
    import torch.distributed as dist
    barrier()
    errs = []
    if flush is None:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            errs.append(step())
            ev[i + 1].record(stream)
        barrier()
        per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        total = ev[0].elapsed_time(ev[-1])
    else:
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush()
            pairs[i][0].record(stream)
            errs.append(step())
            pairs[i][1].record(stream)
        barrier()
        per_step = [a.elapsed_time(b) for a, b in pairs]
        total = sum(per_step)
    return per_step, rank_max(total, torch.device("cuda", torch.cuda.current_device())), errs


L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2


def make_flush(wl, stream, device):
    """An L2 flush for workloads whose inputs fit in L2 (all but the 8 GiB dense A)."""
    import torch
    if wl["kind"] == "dense":
        return None
    buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def flush():
        with torch.cuda.stream(stream):
            buf.fill_(1.0)
    return flush


def l2_note(wl):
    if wl["kind"] == "dense":
        return "inputs larger than L2 (dense A 8 GiB); no flush"
    return "L2 flushed between timed steps (256 MiB write outside the timed event pairs)"


def run_cabs(args):
    import torch
    import torch.distributed as dist

    from paper_1607_07395_gb300 import cabs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    wl = dict(WORKLOADS[args.workload])
    if args.m or args.n:
        # smaller shapes of the same recipe, for profiler captures
        wl["m"], wl["n"] = args.m or wl["m"], args.n or wl["n"]
        wl["desc"] += f" (shape overridden to {wl['m']}x{wl['n']})"
    k, iters = wl["k"], wl["iters"]
    ctx = cabs.Context(local)
    inp = make_inputs(wl, device, seed=1607 + rank)
    src = make_source(cabs, wl, inp)
    samples = wl.get("samples", 0)
    stream = torch.cuda.Stream(device=device)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- the chosen form: B concurrent sketches per step in reduced precision,
    # launched as one captured graph over `lanes` streams, plus each error
    prec = "fp64" if args.workload == "plain" else args.prec
    B = 1 if args.form == "plain" else args.batch
    flags = follow_flags(cabs, args)
    params = [cabs.make_params(wl["m"], wl["n"], k, iters=iters, seed=1607 + rank * 1000 + b, prec=prec,
                               trunc_rtol=trunc_rtol(wl, k), flags=flags,
                               core=wl["core"], err_samples=samples, err_seed=3) for b in range(B)]
    srcs = [src] * B
    outs = [cabs.alloc_result(p, device) for p in params]
    offs, tot = cabs.batched_layout(srcs, params)
    ws = torch.empty(tot + 512, dtype=torch.uint8, device=device)

    def run_batch(lanes, use_graph, srcs_=None):
        # every sketch computes its own relative error (CABS_FLAG_ERROR) on its
        # lane; the B errors are read back to the host once per step
        srcs_ = srcs if srcs_ is None else srcs_
        with torch.cuda.stream(stream):
            if B == 1:
                cabs.cabs_sketch(ctx, srcs_[0], params[0], ws=ws, out=outs[0], stream=stream)
            else:
                cabs.cabs_sketch_batched(ctx, srcs_, params, outs, ws, offs, lanes=lanes, use_graph=use_graph,
                                         stream=stream)
            return torch.cat([o.err for o in outs]).cpu().tolist()

    def step():
        return run_batch(args.lanes, True)

    for _ in range(args.warmup):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    if args.steps <= 0:
        # about two seconds of timed work (enough clock samples), 5 to 2000 steps
        est = max(e0.elapsed_time(e1), 1e-3) if args.warmup > 0 else 50.0
        args.steps = int(rank_max(min(2000, max(5, math.ceil(2000.0 / est))), device))
    sampler = ClockSampler(local)
    launches0 = cabs.cabs_launch_count()
    if B == 1:
        cabs.cabs_profile_read(ctx, reset=True)
        cabs.cabs_profile_enable(ctx, True)
    flush = make_flush(wl, stream, device)
    sampler.start()
    per_step, total_ms, errs = timed_steps(ctx, cabs, step, args.steps, stream, world, barrier, flush)
    clocks = sampler.stop()
    launches = cabs.cabs_launch_count() - launches0
    if B > 1:
        # Per-kernel launch durations of the same batch run serially (one lane,
        # no graph): under concurrent lanes an event pair would also bracket the
        # time a kernel queues behind the other lanes' kernels.
        cabs.cabs_profile_read(ctx, reset=True)
        cabs.cabs_profile_enable(ctx, True)
        timed_steps(ctx, cabs, lambda: run_batch(1, False), args.steps, stream, world, barrier, flush)
    cabs.cabs_profile_enable(ctx, False)
    prof = cabs.cabs_profile_read(ctx, reset=True)
    diag = outs[0].diag()
    sweeps = [diag.sweeps_pilot, diag.sweeps_final]
    all_errs = [e for es in errs for e in es]

    # ---- end to end through the C ABI with host buffers: pinned H2D of the
    # step's inputs, the sketches and their errors, D2H of factors and indices
    e2e = None
    if not args.no_e2e:
        all_cpus = os.sched_getaffinity(0)
        host_cpus = bind_to_gpu_local_cpus(local)
        if wl["kind"] == "rbf":
            hx = torch.from_numpy(inp["X_host"]).pin_memory()
            hy = torch.from_numpy(inp["Y_host"]).pin_memory()
            h2d = hx.numel() * 4 + hy.numel() * 4
        elif wl["kind"] == "csr":
            hcsr = [torch.from_numpy(x).pin_memory() for x in inp["host"]]
            h2d = sum(x.numel() * x.element_size() for x in hcsr)
        else:
            hA = torch.empty(inp["A"].shape, dtype=inp["A"].dtype, pin_memory=True)
            hA.copy_(inp["A"])
            h2d = hA.numel() * hA.element_size()
        outs_host = [[torch.empty(t_.shape, dtype=t_.dtype, pin_memory=True)
                      for t_ in (o.U, o.S, o.V, o.rows, o.cols)] for o in outs]
        d2h = sum(x.numel() * x.element_size() for oh in outs_host for x in oh) + 8 * B  # + the errors

        def e2e_step():
            with torch.cuda.stream(stream):
                if wl["kind"] == "rbf":
                    inp["X"].copy_(hx, non_blocking=True)
                    inp["Y"].copy_(hy, non_blocking=True)
                elif wl["kind"] == "csr":
                    for dst, h in zip((inp["row_ptr"], inp["col_idx"], inp["vals"]), hcsr):
                        dst.copy_(h, non_blocking=True)
                else:
                    inp["A"].copy_(hA, non_blocking=True)
            errs_ = step()  # the step's errors are read back to the host
            with torch.cuda.stream(stream):
                for oh, o in zip(outs_host, outs):
                    for hdst, dsrc in zip(oh, (o.U, o.S, o.V, o.rows, o.cols)):
                        hdst.copy_(dsrc, non_blocking=True)
            return errs_

        e2e_form = "each step: H2D of its inputs, the step, D2H of its results, in order on one stream"
        if wl["kind"] == "dense":
            # Two device copies of A: the next step's H2D runs on a copy stream
            # while this step's sketches run. Every step still copies its whole
            # input from the pinned host buffer inside the timed region (the
            # first copy is ordered after the region's start; each later one
            # waits until the step that last read its buffer has finished).
            A_bufs = [inp["A"], torch.empty_like(inp["A"])]
            srcs_b = [srcs, [cabs.dense_source(A_bufs[1])] * B]
            cstream = torch.cuda.Stream(device)
            copy_done = [torch.cuda.Event(), torch.cuda.Event()]
            compute_done = [torch.cuda.Event(), torch.cuda.Event()]
            st = dict(i=0, K=0)

            def e2e_step():
                i, K = st["i"], st["K"]
                b = i % 2
                if i == 0:
                    cstream.wait_stream(stream)
                    with torch.cuda.stream(cstream):
                        A_bufs[b].copy_(hA, non_blocking=True)
                    copy_done[b].record(cstream)
                if i + 1 < K:
                    nb = 1 - b
                    if i >= 1:
                        cstream.wait_event(compute_done[nb])
                    with torch.cuda.stream(cstream):
                        A_bufs[nb].copy_(hA, non_blocking=True)
                    copy_done[nb].record(cstream)
                stream.wait_event(copy_done[b])
                errs_ = run_batch(args.lanes, True, srcs_b[b])
                compute_done[b].record(stream)
                with torch.cuda.stream(stream):
                    for oh, o in zip(outs_host, outs):
                        for hdst, dsrc in zip(oh, (o.U, o.S, o.V, o.rows, o.cols)):
                            hdst.copy_(dsrc, non_blocking=True)
                st["i"] = i + 1
                return errs_

            # untimed: capture the graphs of both buffers
            st.update(i=0, K=2)
            e2e_step()
            e2e_step()
            torch.cuda.synchronize()
            st.update(i=0, K=args.steps)
            e2e_form = ("each step: H2D of its whole input from pinned memory, the step, D2H of its results; the "
                        "next step's H2D overlaps this step's sketches (two device copies of A, a copy stream)")
        _, e2e_ms, _ = timed_steps(ctx, cabs, e2e_step, args.steps, stream, world, barrier, flush)
        torch.cuda.synchronize()
        if wl["kind"] == "dense":
            del A_bufs, srcs_b
            torch.cuda.empty_cache()
        e2e = dict(value=round(job_value(world, B, args.steps, e2e_ms), 4), unit="sketches/s", form=e2e_form,
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h),
                   host_cpus=f"process bound to the GPU-local CPUs {host_cpus} before the pinned buffers were "
                             f"allocated" if not host_cpus.startswith("unbound") else host_cpus)
        os.sched_setaffinity(0, all_cpus)  # the CPU baseline keeps every core

    # ---- the plain FP32 form on the same GPU, one sketch at a time (comparison)
    plain = None
    if args.form != "plain" and not args.no_plain and args.workload != "plain":
        pp = cabs.make_params(wl["m"], wl["n"], k, iters=iters, seed=1607 + rank * 1000, prec="fp32", core=wl["core"],
                              trunc_rtol=trunc_rtol(wl, k), flags=flags,
                              err_samples=samples, err_seed=3)
        wsp = torch.empty(cabs.cabs_workspace_size(src, pp) + 512, dtype=torch.uint8, device=device)
        outp = cabs.alloc_result(pp, device)

        def pstep():
            with torch.cuda.stream(stream):
                cabs.cabs_sketch(ctx, src, pp, ws=wsp, out=outp, stream=stream)
                return float(outp.err.cpu().item())

        for _ in range(2):
            pstep()
        psteps = max(2, args.steps // 2)
        pper, ptot, perrs = timed_steps(ctx, cabs, pstep, psteps, stream, world, barrier, flush)
        plain = dict(value=round(job_value(world, 1, psteps, ptot), 4), unit="sketches/s",
                     ms_per_sketch=round(ptot / psteps, 4), rel_fro_error=perrs[-1], prec="fp32",
                     form="one sketch per launch sequence, one stream, no graph")

    # ---- the FP64 mode (the paper's arithmetic) at the same configuration, same
    # form (B sketches over the lanes, graph); without the error, whose exact
    # FP64 form costs 2 m n k FP64 flops
    fp64_mode = None
    if prec != "fp64" and not args.no_fp64_mode:
        p64 = [cabs.make_params(wl["m"], wl["n"], k, iters=iters, seed=1607 + rank * 1000 + b, prec="fp64",
                                trunc_rtol=trunc_rtol(wl, k), flags=flags, core=wl["core"]) for b in range(B)]
        o64 = [cabs.alloc_result(q, device) for q in p64]
        off64, tot64 = cabs.batched_layout(srcs, p64)
        ws64 = torch.empty(tot64 + 512, dtype=torch.uint8, device=device)

        def step64():
            with torch.cuda.stream(stream):
                if B == 1:
                    cabs.cabs_sketch(ctx, src, p64[0], ws=ws64, out=o64[0], stream=stream)
                else:
                    cabs.cabs_sketch_batched(ctx, srcs, p64, o64, ws64, off64, lanes=args.lanes, use_graph=True,
                                             stream=stream)
            return []

        step64()
        torch.cuda.synchronize()
        n64 = 2
        _, t64, _ = timed_steps(ctx, cabs, step64, n64, stream, world, barrier, flush)
        fp64_mode = dict(value=round(job_value(world, B, n64, t64), 4), unit="sketches/s", steps=n64,
                         ms_per_step=round(t64 / n64, 3), prec="fp64", error_included=False,
                         form=f"{B} sketches over {args.lanes if B > 1 else 1} lanes, graph; no error")
        del ws64, o64
        torch.cuda.empty_cache()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    peaks = load_peaks()
    alu = measure_alu_peaks(device)  # after the timed region
    peaks.update({k_: v for k_, v in alu.items() if k_.endswith("_tflops")})
    eb = 8 if prec == "fp64" else 4
    roof, table, roof_next = roofline(prof, wl, k, iters, eb, sweeps, args.steps * B, peaks, prec,
                                      args.workload if not (args.m or args.n) else None,
                                      [diag.refine_pilot, diag.refine_final])
    gather = None
    if wl["kind"] in ("dense", "plain") and "gather_cols_kernel" in prof:
        gl, gms = prof["gather_cols_kernel"]
        rl, rms = prof.get("gather_rows_t_kernel", (0, 0.0))
        m, n = wl["m"], wl["n"]
        nsk = args.steps * B
        useful = nsk * 2 * ((m * k + n * k) * eb + k * k * eb)
        sectors = nsk * 2 * (m * k * 32 + n * k * eb)
        secs = (gms + rms) / 1e3
        gather = dict(useful_gbs=round(useful / secs / 1e9, 2), dram_sector_gbs=round(sectors / secs / 1e9, 2),
                      frac_of_hbm=round(sectors / secs / 1e9 / peaks["hbm_gbs"], 4),
                      ms_per_sketch=round((gms + rms) / nsk, 4))
    lat = sorted(per_step)
    res = dict(metric=METRIC, value=round(job_value(world, B, args.steps, total_ms), 4), unit="sketches/s",
               n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=round(total_ms / args.steps, 4),
               higher_is_better=True, scaling="weak", vs_baseline=None,
               dtype={"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[prec] + "+f64core",
               data="synthetic",
               config=dict(workload=args.workload, desc=wl["desc"], m=wl["m"], n=wl["n"], k=k, iters=iters,
                           prec=prec, core=wl["core"], trunc_rtol=trunc_rtol(wl, k), form=args.form,
                           follow=args.follow, svd_form=bool(args.svd_form),
                           sketches_per_step=B,
                           lanes=args.lanes if B > 1 else 1, graph=B > 1,
                           parallelism=f"replicas x{world}",
                           l2=l2_note(wl)),
               latency_ms=dict(step_p50=round(statistics.median(per_step), 4),
                               step_p99=round(lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)], 4)),
               rel_fro_error=dict(median=statistics.median(all_errs), max=max(all_errs)),
               gpu_launches=int(launches),
               diag=dict(svd_sweeps=sweeps, svd_refine=[diag.refine_pilot, diag.refine_final],
                         svd_status=int(diag.status), rank=[diag.rank_pilot, diag.rank_final],
                         snap_fallbacks=int(diag.snap_fallbacks), rechecked=int(diag.rechecked)),
               roofline=roof, roofline_next=roof_next, kernels=table,
               kernel_timing=("serial profiled pass of the same batch after the timed region" if B > 1
                              else "timed region"),
               gather=gather, plain_fp32=plain, fp64_mode=fp64_mode, e2e=e2e, clocks=clocks,
               peaks=dict(hbm_gbs=peaks["hbm_gbs"], bf16_tflops=peaks["bf16_tflops"],
                          bf16_tflops_sustained=peaks["bf16_tflops_sustained"], source=peaks["source"],
                          measured_here=alu, derived_fp32_tflops=round(FP32_PEAK_TFLOPS, 2),
                          derived_fp64_tflops=round(FP64_PEAK_TFLOPS, 3)))
    if wl["kind"] == "dense" and "L" in inp:
        res["rel_fro_error_noiseless"] = noiseless_error(inp["L"], outs[0])
    if wl["kind"] != "plain" and not (args.m or args.n) and not args.no_precision:
        res["precision"] = precision_excess(cabs, ctx, wl, device)
    if not args.no_cpu:
        res["cpu_baseline"] = run_cpu_baseline(args.workload, args.cpu_steps)
        if "precision" in res and res["cpu_baseline"].get("oracle_error") is not None:
            res["precision"]["oracle_fp64"] = res["cpu_baseline"]["oracle_error"]
    if world > 1:
        dist.destroy_process_group()
    return res


def follow_flags(cabs, args):
    """cabs_params flags of the follow-up variant (Section 5: (d) weighted
    k-means, (e) leverage scores, (f) hard threshold) and the SVD-form output
    (supplementary Section 3)."""
    f = {"kmeans": 0, "threshold": cabs.FLAG_HARD_THRESHOLD, "leverage": cabs.FLAG_LEVERAGE}[args.follow]
    return f | (cabs.FLAG_SVD_FORM if args.svd_form else 0)


def run_sketch_cur(args):
    """Sketch-CUR (Section 2.2, Algorithm 1; Section 5 comparison (a)) on the
    workload's matrix: kb base and kt = 3 kb target samples per side; B
    sketches per step on B streams (one workspace each)."""
    import torch

    from paper_1607_07395_gb300 import cabs
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    wl = dict(WORKLOADS[args.workload])
    kb = args.kb or max(1, min(wl["k"], cabs.MAX_K) // 3)
    kt = min(3 * kb, cabs.MAX_K, wl["m"], wl["n"])
    prec = "fp64" if args.workload == "plain" else "fp32"
    ctx = cabs.Context(local)
    inp = make_inputs(wl, device, seed=1607 + rank)
    src = make_source(cabs, wl, inp)
    B = 1 if args.form == "plain" else args.batch
    streams = [torch.cuda.Stream(device=device) for _ in range(B)]
    ps = [cabs.make_cur_params(wl["m"], wl["n"], kb, kt, seed=1607 + rank * 1000 + b, prec=prec,
                               trunc_rtol=trunc_rtol(wl, max(kb, kt))) for b in range(B)]
    outs = [cabs.cabs_sketch_cur(ctx, src, p, stream=st) for p, st in zip(ps, streams)]
    main = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def step():
        ev = torch.cuda.Event()
        ev.record(main)
        for p, st, o in zip(ps, streams, outs):
            st.wait_event(ev)
            cabs.cabs_sketch_cur(ctx, src, p, stream=st, ws=o.ws)
        for st in streams:
            main.wait_stream(st)
        return []

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    if args.steps <= 0:
        t0 = time.time()
        step()
        torch.cuda.synchronize()
        est = max((time.time() - t0) * 1e3, 1e-3)
        args.steps = int(rank_max(min(2000, max(5, math.ceil(2000.0 / est))), device))
    sampler = ClockSampler(local)
    launches0 = cabs.cabs_launch_count()
    sampler.start()
    per_step, total_ms, _ = timed_steps(ctx, cabs, step, args.steps, main, world, barrier,
                                        make_flush(wl, main, device))
    clocks = sampler.stop()
    launches = cabs.cabs_launch_count() - launches0
    cabs.cabs_profile_read(ctx, reset=True)
    cabs.cabs_profile_enable(ctx, True)
    for p, o in zip(ps, outs):
        cabs.cabs_sketch_cur(ctx, src, p, stream=main, ws=o.ws)
    torch.cuda.synchronize()
    cabs.cabs_profile_enable(ctx, False)
    prof = cabs.cabs_profile_read(ctx, reset=True)
    samples = wl.get("samples", 0)
    sp = cabs.make_params(wl["m"], wl["n"], kb, prec=prec)
    errs = [cabs.cabs_error(ctx, src, sp, o, samples=samples, seed=3) for o in outs]
    if rank != 0:
        return None
    total = sum(x[1] for x in prof.values())
    table = {nm: dict(launches=l, total_ms=round(t, 4), share=round(t / total, 4))
             for nm, (l, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    top = next(iter(table))
    K = max(kb, kt)
    roof = None
    if top.startswith("svd32"):
        # FP32 Jacobi on the K x K padded C_bar and R_bar: 18 K flops per column pair per sweep
        rk = [int(x) for x in outs[0].ranks.tolist()]
        l, t = prof[top]
        fl = sum(sw * (K * (K - 1) / 2) * 18.0 * K for sw in rk[2:4])
        ach = fl / (t / max(l, 1) * 2 / 1e3) / 1e12  # two SVD launches per sketch
        roof = dict(kernel=top, bound="alu", achieved=round(ach, 4), peak=round(FP32_PEAK_TFLOPS, 3),
                    unit="TFLOP/s", frac=round(ach / FP32_PEAK_TFLOPS, 5), traffic=None,
                    avg_launch_ms=round(t / max(l, 1), 5), peak_source="derived from unit counts x 2.07 GHz",
                    note=f"FP32 Jacobi of a {K} x {K} matrix on one 16-CTA cluster: latency-bound")
    return dict(metric=METRIC, value=round(job_value(world, B, args.steps, total_ms), 4), unit="sketches/s",
                n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=round(total_ms / args.steps, 4),
                higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={"fp64": "f64", "fp32": "f32"}[prec] + "+f64core", data="synthetic",
                config=dict(workload=args.workload, algo="sketch_cur", desc=wl["desc"], m=wl["m"], n=wl["n"],
                            kb=kb, kt=kt, prec=prec, sketches_per_step=B, streams=B,
                            parallelism=f"replicas x{world}"),
                latency_ms=dict(step_p50=round(statistics.median(per_step), 4)),
                rel_fro_error=dict(median=statistics.median(errs), max=max(errs),
                                   samples=samples or "exact"),
                ranks=[int(x) for x in outs[0].ranks.tolist()[:2]],
                svd_sweeps=[int(x) for x in outs[0].ranks.tolist()[2:4]], gpu_launches=int(launches),
                roofline=roof, kernels=table, clocks=clocks, e2e=None,
                e2e_note="Sketch-CUR is a comparison row: device-resident inputs only")


def run_oracle_full(args):
    """The oracle once on the whole dense workload (65536 x 32768, k = 256, c = 5,
    stabilised core, trunc k 2^-24) on the host, beside the GPU's FP64-mode
    sketch of the same matrix and seed: pilot and follow-up indices compared
    bit for bit, U S V^T on 64 sampled rows, and both exact errors. One JSON
    line; minutes of host time (not part of the default run)."""
    import numpy as np
    import torch

    from oracle import cabs_ref as o
    from paper_1607_07395_gb300 import cabs
    wl = WORKLOADS["dense"]
    device = torch.device("cuda", 0)
    inp = make_inputs(wl, device, seed=1607)
    A = inp["A"]
    k = wl["k"]
    tr = trunc_rtol(wl, k)
    ctx = cabs.Context(0)
    src = cabs.dense_source(A)
    p = cabs.make_params(wl["m"], wl["n"], k, iters=wl["iters"], seed=1607, prec="fp64", core=wl["core"],
                         trunc_rtol=tr, err_samples=0, err_seed=3)
    t0 = time.perf_counter()
    sk = cabs.cabs_sketch(ctx, src, p)
    torch.cuda.synchronize()
    gpu_s = time.perf_counter() - t0
    gpu_err = float(sk.err.cpu().item())
    Ah = A.cpu().numpy()
    del inp
    t0 = time.perf_counter()
    ref = o.cabs(o.DenseSource(Ah), k, iters=wl["iters"], seed=1607, mode=wl["core"], trunc_rtol=tr)
    t1 = time.perf_counter()
    ref_err = o.rel_fro_error_dense(Ah, ref.final.U, ref.final.S, ref.final.V)
    t2 = time.perf_counter()
    rows = np.arange(0, wl["m"], wl["m"] // 64)
    U, S, V = (t.cpu().numpy() for t in (sk.U, sk.S, sk.V))
    got = (U[rows] * S) @ V.T
    want = (ref.final.U[rows] * ref.final.S) @ ref.final.V.T
    return dict(workload="dense 65536x32768 FP32, k=256, c=5, stabilised, trunc k 2^-24, seed 1607",
                threads=int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
                oracle_sketch_s=round(t1 - t0, 2), oracle_error_s=round(t2 - t1, 2), oracle_error=ref_err,
                gpu_fp64_error=gpu_err, gpu_fp64_sketch_and_error_s=round(gpu_s, 3),
                error_rel_diff=abs(gpu_err - ref_err) / ref_err,
                pilot_rows_equal=sk.pilot_rows.cpu().numpy().tolist() == ref.pilot_rows.tolist(),
                pilot_cols_equal=sk.pilot_cols.cpu().numpy().tolist() == ref.pilot_cols.tolist(),
                rows_equal=sk.rows.cpu().numpy().tolist() == ref.rows.tolist(),
                cols_equal=sk.cols.cpu().numpy().tolist() == ref.cols.tolist(),
                factors_rel_diff_sampled_rows=float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                rank=[int(ref.pilot.rank), int(ref.final.rank)])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cb = run_cpu_baseline(args.workload, max(1, args.steps))
    cb["value"] = round(cb["value"], 6)  # the line's value, as the cpu_baseline of this run
    wl = WORKLOADS[args.workload]
    return dict(metric=METRIC, value=cb["value"], unit="sketches/s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(cb["seconds_per_sketch_extrapolated"] * 1e3, 3),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=args.workload, desc=wl["desc"], m=wl["m"], n=wl["n"], k=wl["k"],
                            iters=wl["iters"], prec="fp64", core=wl["core"], parallelism="cpu"),
                cpu_baseline=cb, e2e=dict(value=round(cb["value"], 6), unit="sketches/s", h2d_bytes_per_step=0,
                                          d2h_bytes_per_step=0))


def run_systems(args):
    """The batched (uneven sizes, one graph) and serving (Poisson stream) workloads."""
    if args.impl == "reference":
        return dict(impl="reference", unavailable="the oracle baseline is timed on the dense, RBF and plain "
                                                  "workloads; for these the comparison is the plain FP32 form")
    import torch
    import torch.distributed as dist

    import bench_systems as bs
    from paper_1607_07395_gb300 import cabs
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    ctx = cabs.Context(local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    if args.workload == "batched":
        r = bs.run_batched(args, cabs, torch, device, ctx, timed_steps, barrier, ClockSampler, job_value)
    else:
        r = bs.run_serve(args, cabs, torch, device, ctx, ClockSampler)
    if world > 1:
        v = rank_max(1.0 / r["value"] if r["value"] else float("inf"), device)
        r["value"] = round(world / v, 4) if v and v != float("inf") else None
        dist.destroy_process_group()
    if rank != 0:
        return None
    out = dict(metric=METRIC, value=r["value"], unit="sketches/s", n_gpus=world, steps=r["steps"],
               warmup=args.warmup, ms_per_step=r["ms_per_step"], higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype={"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.prec] +
               "+f64core", data="synthetic", config=dict(r["config"], parallelism=f"replicas x{world}"),
               latency_ms=r["latency_ms"], rel_fro_error=r["rel_fro_error"], plain_fp32=r["plain_fp32"],
               gpu_launches=r.get("gpu_launches"), clocks=r["clocks"],
               e2e=None, e2e_note="inputs stay resident by design (serving keeps its matrices and factors in HBM)")
    for key in ("fixed", "autotune", "no_graph", "per_kind", "capacity", "overlap"):
        if key in r:
            out[key] = r[key]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: about 2 s of timed work)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cabs", choices=["cabs", "reference"])
    ap.add_argument("--workload", default="dense", choices=sorted(WORKLOADS) + ["batched", "serve"],
                    help="batched: 512 uneven dense sketches per graph; serve: a 200/s Poisson request stream")
    ap.add_argument("--prec", default="bf16", choices=["fp32", "tf32", "bf16", "fp64"])
    ap.add_argument("--form", default="batched", choices=["batched", "plain"],
                    help="batched: --batch concurrent sketches per step over --lanes streams (captured graph)")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lanes", type=int, default=8)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--m", type=int, default=0, help="override the workload's rows (profiler captures)")
    ap.add_argument("--n", type=int, default=0, help="override the workload's columns (profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the per-mode error report on the slice")
    ap.add_argument("--no-fp64-mode", action="store_true", help="skip the FP64-mode throughput leg")
    ap.add_argument("--oracle-full", action="store_true",
                    help="run the oracle once on the whole dense workload beside the GPU FP64 sketch (minutes)")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--batch-count", type=int, default=512, help="members of the batched workload")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="measured seconds of the serving workload")
    ap.add_argument("--follow", default="kmeans", choices=["kmeans", "threshold", "leverage"],
                    help="follow-up sampling: weighted k-means (Algorithm 2), or the leverage-score or "
                         "hard-threshold variants of Section 5")
    ap.add_argument("--svd-form", action="store_true", help="return every sketch in SVD form (orthogonalised)")
    ap.add_argument("--algo", default="cabs", choices=["cabs", "sketch_cur"],
                    help="cabs (Algorithm 2) or the Sketch-CUR comparison (Algorithm 1, target = 3 x base)")
    ap.add_argument("--kb", type=int, default=0, help="Sketch-CUR base samples (default k / 3)")
    ap.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args.workload, args.steps)
        return
    if args.oracle_full:
        res = run_oracle_full(args)
    elif args.workload in ("batched", "serve"):
        res = run_systems(args)
    elif args.impl == "reference":
        res = run_reference(args)
    elif args.algo == "sketch_cur":
        res = run_sketch_cur(args)
    else:
        res = run_cabs(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
