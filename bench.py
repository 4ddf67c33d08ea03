"""Benchmark of the CABS hot path (one sketch + its error per step) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cabs|reference]
                    [--workload dense|rbf|plain] [--prec fp32|tf32|bf16|fp64]

A step is one pass of the whole hot path over one synthetic input: pilot
draw, gathers, FP64 core, embeddings, weighted k-means on both sides, snap,
follow-up gather and core (Algorithm 2), then the relative Frobenius error
(exact for dense inputs, 10^6 sampled entries for the implicit RBF matrix).
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

WORKLOADS = {
    # BASELINE configuration 3: dense stored FP32 A, 65536 x 32768 (8 GiB)
    "dense": dict(kind="dense", m=65536, n=32768, rank=256, k=256, iters=5, core="stabilized",
                  desc="dense FP32 A 65536x32768 = U diag(exp(-i/30)) V^T (rank 256) + N(0,1e-4^2); k=256, c=5"),
    # BASELINE configuration 2: implicit RBF matrix, 1e5 x 1e5 points in d=16
    "rbf": dict(kind="rbf", m=100000, n=100000, d=16, k=200, iters=10, core="pinv", samples=1000000,
                desc="implicit RBF exp(-|x-y|^2/2s^2), 1e5 x 1e5 points d=16 (50-comp. mixture); k=200, c=10"),
    # BASELINE configuration 1: plain FP64 2000 x 1500
    "plain": dict(kind="plain", m=2000, n=1500, k=20, iters=5, core="pinv",
                  desc="plain FP64 A 2000x1500 = U V^T + N(0,1e-6); k=20, c=5"),
}

# Peaks: measured copy bandwidth and BF16 GEMM from MEASURED_PEAKS.json; the
# FP32 / FP64 CUDA-core peaks are derived from unit counts and the maximum
# clock (152 SMs x 128 FP32 lanes or 2 FP64 lanes x 2 flops x 2.07 GHz).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


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
        A, _, _, _ = synth.decaying_lowrank_device(wl["m"], wl["n"], rank=wl["rank"], seed=seed, device=device)
        return dict(A=A)
    if wl["kind"] == "rbf":
        X, Y, sig = synth.rbf_mixture(wl["m"], wl["n"], d=wl["d"], seed=seed)
        return dict(X=torch.from_numpy(X).to(device), Y=torch.from_numpy(Y).to(device), sigma=float(sig),
                    X_host=X, Y_host=Y)
    A = synth.plain_lowrank(wl["m"], wl["n"], seed=seed)
    return dict(A=torch.from_numpy(np.ascontiguousarray(A)).to(device))


def make_source(cabs, wl, inp):
    if wl["kind"] == "rbf":
        return cabs.rbf_source(inp["X"], inp["Y"], inp["sigma"])
    return cabs.dense_source(inp["A"])


# ------------------------------------------------------- algorithmic units

def algorithmic(name, wl, k, iters, elem_bytes, svd_sweeps):
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
    if name == "snap_cand_kernel":
        return "alu", 3.0 * (m + n) * k * d, "TFLOP/s", 2
    if name.startswith("extrap_gemm_kernel"):
        side = m if "C V_w" in name else n
        return "alu", 2 * 2.0 * side * k * k, "TFLOP/s", 2
    if name in ("rbf_block_kernel(C)", "rbf_block_kernel(Rt)"):
        side = m if name.endswith("(C)") else n
        return "alu", 2 * side * k * (3.0 * wl.get("d", 16) + 20), "TFLOP/s", 2
    if name == "update_kernel":
        return "hbm", iters * (m + n) * d * elem_bytes, "GB/s", 2 * iters
    return None


def roofline(prof, wl, k, iters, elem_bytes, svd_sweeps, steps, peaks, prec):
    """Roofline of the kernel with the largest device time in the timed region."""
    if not prof:
        return None, None
    name, (launches, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    info = algorithmic(name, wl, k, iters, elem_bytes, svd_sweeps)
    table = {nm: dict(launches=l, total_ms=round(t, 4), share=round(t / sum(x[1] for x in prof.values()), 4))
             for nm, (l, t) in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    if info is None:
        return dict(kernel=name, bound=None, achieved=None, peak=None, unit=None, frac=None, traffic=None), table
    bound, amount, unit, _ = info
    secs = ms / 1e3
    achieved = amount * steps / secs / (1e12 if unit == "TFLOP/s" else 1e9)
    if bound == "hbm":
        peak, src = peaks["hbm_gbs"], peaks["source"] + " copy"
    elif bound == "tensor":
        peak = peaks["bf16_tflops_sustained"] if prec == "bf16" else peaks["bf16_tflops_sustained"] / 2
        src = peaks["source"] + (" bf16 sustained" if prec == "bf16" else " bf16 sustained / 2 (tf32 nominal ratio)")
    else:
        fp64 = name in ("svd_jacobi_kernel", "refine_persistent_kernel") or (prec == "fp64" and not name.startswith("svd32"))
        peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
        src = "derived from unit counts x 2.07 GHz"
    return dict(kernel=name, bound=bound, achieved=round(achieved, 4), peak=round(peak, 3), unit=unit,
                frac=round(achieved / peak, 5), traffic=None, peak_source=src,
                avg_launch_ms=round(ms / max(launches, 1), 5)), table


# ------------------------------------------------------------------ clocks

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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
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
    else:
        A = synth.plain_lowrank(s["m"], s["n"], seed=1607)
        src = o.DenseSource(A)
    times = []
    for step in range(steps):
        t0 = time.perf_counter()
        r = o.cabs(src, s["k"], iters=s["iters"], seed=1607 + step, mode=wl["core"])
        t1 = time.perf_counter()
        if wl["kind"] == "rbf":
            err = o.rel_fro_error_sampled(src, r.final.U, r.final.S, r.final.V, 3, s["samples"])
        else:
            err = o.rel_fro_error_dense(src.A, r.final.U, r.final.S, r.final.V)
        t2 = time.perf_counter()
        times.append((t1 - t0) * s["scale_sketch"] + (t2 - t1) * s["scale_err"])
    print(json.dumps(dict(times=times, err=err, sample=s)))


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
                seconds_per_sketch_extrapolated=per)


# --------------------------------------------------------------- GPU arm

def run_cabs(args):
    import torch
    import torch.distributed as dist

    from paper_1607_07395_gb300 import cabs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local)) if "device_id" in \
            dist.init_process_group.__code__.co_varnames else dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    prec = "fp64" if args.workload == "plain" else args.prec
    k, iters = wl["k"], wl["iters"]
    ctx = cabs.Context(local)
    inp = make_inputs(wl, device, seed=1607 + rank)
    src = make_source(cabs, wl, inp)
    p = cabs.make_params(wl["m"], wl["n"], k, iters=iters, seed=1607 + rank, prec=prec, core=wl["core"])
    ws = torch.empty(cabs.cabs_workspace_size(src, p) + 512, dtype=torch.uint8, device=device)
    out = cabs.alloc_result(p, device)
    samples = wl.get("samples", 0)
    stream = torch.cuda.current_stream()

    def step():
        sk = cabs.cabs_sketch(ctx, src, p, ws=ws, out=out, stream=stream)
        return cabs.cabs_error(ctx, src, p, sk, samples=samples, seed=3, stream=stream)

    for _ in range(args.warmup):
        err = step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    cabs.cabs_profile_read(ctx, reset=True)
    cabs.cabs_profile_enable(ctx, True)
    launches0 = cabs.cabs_launch_count()
    barrier()
    sampler.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    errs = []
    for i in range(args.steps):
        errs.append(step())
        ev[i + 1].record(stream)
    barrier()
    clocks = sampler.stop()
    launches = cabs.cabs_launch_count() - launches0
    cabs.cabs_profile_enable(ctx, False)
    prof = cabs.cabs_profile_read(ctx, reset=True)
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    diag = out.diag()
    sweeps = [diag.sweeps_pilot, diag.sweeps_final]

    # end to end through the C ABI with host buffers: pinned H2D of the
    # step's inputs, the sketch and its error, D2H of the factors and indices
    e2e = None
    if not args.no_e2e:
        if wl["kind"] == "rbf":
            hx = torch.from_numpy(inp["X_host"]).pin_memory()
            hy = torch.from_numpy(inp["Y_host"]).pin_memory()
            h2d = hx.numel() * 4 + hy.numel() * 4
        else:
            hA = torch.empty(inp["A"].shape, dtype=inp["A"].dtype, pin_memory=True)
            hA.copy_(inp["A"])
            h2d = hA.numel() * hA.element_size()
        outs_host = [torch.empty(t_.shape, dtype=t_.dtype, pin_memory=True)
                     for t_ in (out.U, out.S, out.V, out.rows, out.cols)]
        d2h = sum(x.numel() * x.element_size() for x in outs_host) + 8
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            if wl["kind"] == "rbf":
                inp["X"].copy_(hx, non_blocking=True)
                inp["Y"].copy_(hy, non_blocking=True)
            else:
                inp["A"].copy_(hA, non_blocking=True)
            step()  # the error is read back to the host inside cabs_error
            for hdst, dsrc in zip(outs_host, (out.U, out.S, out.V, out.rows, out.cols)):
                hdst.copy_(dsrc, non_blocking=True)
        e1.record(stream)
        barrier()
        e2e_ms = e0.elapsed_time(e1)
        te = torch.tensor([e2e_ms], dtype=torch.float64, device=device)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = dict(value=round(world * args.steps / (float(te.item()) / 1e3), 4), unit="sketches/s",
                   h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h))

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    peaks = load_peaks()
    eb = 8 if prec == "fp64" else 4
    roof, table = roofline(prof, wl, k, iters, eb, sweeps, args.steps, peaks, prec)
    gather = None
    if wl["kind"] in ("dense", "plain") and "gather_cols_kernel" in prof:
        gl, gms = prof["gather_cols_kernel"]
        rl, rms = prof.get("gather_rows_t_kernel", (0, 0.0))
        m, n = wl["m"], wl["n"]
        useful = args.steps * 2 * ((m * k + n * k) * eb + k * k * eb)
        sectors = args.steps * 2 * (m * k * 32 + n * k * eb)
        secs = (gms + rms) / 1e3
        gather = dict(useful_gbs=round(useful / secs / 1e9, 2), dram_sector_gbs=round(sectors / secs / 1e9, 2),
                      frac_of_hbm=round(sectors / secs / 1e9 / peaks["hbm_gbs"], 4), ms_per_step=round(
                          (gms + rms) / args.steps, 4))
    res = dict(metric=METRIC, value=round(world * args.steps / (total_ms / 1e3), 4), unit="sketches/s",
               n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=round(total_ms / args.steps, 4),
               higher_is_better=True, scaling="weak", vs_baseline=None,
               dtype={"fp64": "f64", "fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[prec] + "+f64core",
               data="synthetic",
               config=dict(workload=args.workload, desc=wl["desc"], m=wl["m"], n=wl["n"], k=k, iters=iters,
                           prec=prec, core=wl["core"], parallelism=f"replicas x{world}",
                           l2="inputs larger than L2 (dense A 8 GiB)" if wl["kind"] == "dense" else
                           "entries generated on the fly; factors and points re-read each step"),
               latency_ms=dict(p50=round(statistics.median(per_step), 4),
                               p99=round(sorted(per_step)[min(len(per_step) - 1,
                                                              int(math.ceil(0.99 * len(per_step))) - 1)], 4)),
               rel_fro_error=errs[-1], gpu_launches=int(launches),
               diag=dict(svd_sweeps=sweeps, svd_status=int(diag.status), rank=[diag.rank_pilot, diag.rank_final],
                         snap_fallbacks=int(diag.snap_fallbacks), rechecked=int(diag.rechecked)), roofline=roof, kernels=table, gather=gather,
               e2e=e2e, clocks=clocks)
    if not args.no_cpu:
        res["cpu_baseline"] = run_cpu_baseline(args.workload, args.cpu_steps)
    if world > 1:
        dist.destroy_process_group()
    return res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cb = run_cpu_baseline(args.workload, max(1, args.steps))
    wl = WORKLOADS[args.workload]
    return dict(metric=METRIC, value=round(cb["value"], 6), unit="sketches/s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(cb["seconds_per_sketch_extrapolated"] * 1e3, 3),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=args.workload, desc=wl["desc"], m=wl["m"], n=wl["n"], k=wl["k"],
                            iters=wl["iters"], prec="fp64", core=wl["core"], parallelism="cpu"),
                cpu_baseline=cb, e2e=dict(value=round(cb["value"], 6), unit="sketches/s", h2d_bytes_per_step=0,
                                          d2h_bytes_per_step=0))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cabs", choices=["cabs", "reference"])
    ap.add_argument("--workload", default="dense", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="fp32", choices=["fp32", "tf32", "bf16", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--cpu-worker", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args.workload, args.steps)
        return
    if args.impl == "reference":
        res = run_reference(args)
    else:
        res = run_cabs(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
