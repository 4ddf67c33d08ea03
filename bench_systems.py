"""The two systems workloads of bench.py (imported by it; not run alone).

batched  512 independent dense FP32 sketches of uneven size, one captured
         graph per step (`cabs_sketch_batched`): m, n ~ U[1000, 20000], rank ~
         U[10, 100], k ~ U[16, 128], each matrix built like the dense workload
         (U diag(exp(-i/30)) V^T + N(0, 1e-4^2)). Each member also computes its
         exact relative error. The fixed form (16 lanes, default launch shapes)
         is timed first; then `cabs_autotune` picks the launch shapes per shape
         bucket and the lanes from timed trials, and the tuned form is the
         line's value. Compared with the same members run one by one in FP32
         (one launch sequence each, no graph).
serve    continuous batching (`cabs_serve_*`): a Poisson stream of requests at
         200 per second for 60 s after a 5 s warm-up, admitted by HBM footprint
         into a fixed arena, their factors kept resident until read. The mix:
         50 % dense requests on a pool of 32 resident matrices from the batched
         distribution, 45 % implicit RBF requests (m = n in [10^4, 2 10^5],
         k in [32, 256], 10^5 sampled entries for the error), 5 % plain FP64
         2000 x 1500 requests. Latency is submit-to-completion; p50 / p99 and
         throughput are reported, beside the plain FP32 form (the same request
         sequence served one at a time, back to back).
"""
from __future__ import annotations

import math
import statistics
import time

import numpy as np


def _pct(v, q):
    s = sorted(v)
    return s[min(len(s) - 1, max(0, int(math.ceil(q * len(s))) - 1))]


def batched_members(cabs, torch, device, count, seed, prec):
    """Sources and params of the uneven batch (FP32 matrices resident in HBM)."""
    from workloads import synth
    specs = synth.batched_specs(count, seed=seed)
    need = sum(s["m"] * s["n"] * 4 for s in specs)
    free, _ = torch.cuda.mem_get_info(device)
    if need > 0.8 * free:  # keep room for workspaces and factors
        raise RuntimeError(f"the {count} batched matrices need {need / 2**30:.1f} GiB; {free / 2**30:.1f} GiB free")
    srcs, params, mats = [], [], []
    for i, s in enumerate(specs):
        A, _, _, _ = synth.decaying_lowrank_device(s["m"], s["n"], rank=s["rank"], seed=seed + 17 * i, device=device,
                                                   noise_fp32=True)
        mats.append(A)
        srcs.append(cabs.dense_source(A))
        params.append(cabs.make_params(s["m"], s["n"], s["k"], iters=5, seed=seed + i, prec=prec, core="stabilized",
                                       trunc_rtol=s["k"] * 2.0 ** -24,
                                       err_samples=0, err_seed=3))
    return specs, srcs, params, mats


def run_batched(args, cabs, torch, device, ctx, timed_steps, barrier, ClockSampler, job_value):
    count = args.batch_count
    specs, srcs, params, mats = batched_members(cabs, torch, device, count, 1607, args.prec)
    outs = [cabs.alloc_result(p, device) for p in params]
    offs, tot = cabs.batched_layout(srcs, params)
    ws = torch.empty(tot + 512, dtype=torch.uint8, device=device)
    stream = torch.cuda.Stream(device=device)
    lanes = 16

    def step():
        with torch.cuda.stream(stream):
            cabs.cabs_sketch_batched(ctx, srcs, params, outs, ws, offs, lanes=lanes, use_graph=True, stream=stream)
            return torch.cat([o.err for o in outs]).cpu().tolist()

    steps = args.steps if args.steps > 0 else 3

    def step_nograph():
        with torch.cuda.stream(stream):
            cabs.cabs_sketch_batched(ctx, srcs, params, outs, ws, offs, lanes=16, use_graph=False, stream=stream)
            return torch.cat([o.err for o in outs]).cpu().tolist()

    # the same batch launched kernel by kernel (no graph): what launch overhead costs
    step_nograph()
    torch.cuda.synchronize()
    _, nograph_ms, _ = timed_steps(ctx, cabs, step_nograph, steps, stream, 1, barrier)
    # fixed form: 16 lanes, default launch shapes
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    _, fixed_ms, _ = timed_steps(ctx, cabs, step, steps, stream, 1, barrier)
    # autotuner (untimed): launch shapes per bucket and the lanes
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        tuned_lanes = cabs.cabs_autotune(ctx, srcs, params, outs, ws, offs, stream=stream)
    tune_s = time.perf_counter() - t0
    shapes = {}
    for p in params:
        sh, _ = cabs.cabs_tune_get(ctx, p)
        key = f"k<={((p.k2 + 31) // 32) * 32},m+n~2^{int(math.log2(p.m + p.n))}"
        shapes[key] = sh
    lanes = 0  # the autotuner's lanes
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(device.index or 0)
    l0 = cabs.cabs_launch_count()
    sampler.start()
    per_step, total_ms, errs = timed_steps(ctx, cabs, step, steps, stream, 1, barrier)
    clocks = sampler.stop()
    launches = cabs.cabs_launch_count() - l0
    all_errs = [e for es in errs for e in es]

    # the plain FP32 form: the same members one at a time, no graph
    pparams = [cabs.make_params(s["m"], s["n"], s["k"], iters=5, seed=1607 + i, prec="fp32", core="stabilized",
                                trunc_rtol=s["k"] * 2.0 ** -24,
                                err_samples=0, err_seed=3) for i, s in enumerate(specs)]
    pws = torch.empty(max(cabs.cabs_workspace_size(s, p) for s, p in zip(srcs, pparams)) + 512, dtype=torch.uint8,
                      device=device)
    pouts = [cabs.alloc_result(p, device) for p in pparams]

    def pstep():
        with torch.cuda.stream(stream):
            for s, p, o in zip(srcs, pparams, pouts):
                cabs.cabs_sketch(ctx, s, p, ws=pws, out=o, stream=stream)
            return torch.cat([o.err for o in pouts]).cpu().tolist()

    pstep()
    _, ptot, perrs = timed_steps(ctx, cabs, pstep, 1, stream, 1, barrier)
    total_bytes = sum(s["m"] * s["n"] * 4 for s in specs)
    return dict(value=round(job_value(1, count, steps, total_ms), 4), steps=steps,
                ms_per_step=round(total_ms / steps, 4), gpu_launches=int(launches), clocks=clocks,
                latency_ms=dict(step_p50=round(statistics.median(per_step), 4), step_p99=round(_pct(per_step, 0.99), 4)),
                rel_fro_error=dict(median=statistics.median(all_errs), max=max(all_errs)),
                fixed=dict(value=round(job_value(1, count, steps, fixed_ms), 4), unit="sketches/s", lanes=16,
                           shapes="defaults"),
                no_graph=dict(value=round(job_value(1, count, steps, nograph_ms), 4), unit="sketches/s", lanes=16,
                              launches_per_step=int(launches / steps),
                              form="the same batch launched kernel by kernel over 16 lanes, no graph"),
                autotune=dict(seconds=round(tune_s, 2), lanes=tuned_lanes, buckets=len(shapes), shapes=shapes),
                plain_fp32=dict(value=round(count / (ptot / 1e3), 4), unit="sketches/s",
                                rel_fro_error=dict(median=statistics.median(perrs[0]), max=max(perrs[0])),
                                form="one sketch per launch sequence, one stream, no graph"),
                config=dict(workload="batched", members=count, lanes=tuned_lanes, graph=True, prec=args.prec,
                            shapes="autotuned",
                            core="stabilized", matrices_gib=round(total_bytes / 2**30, 1),
                            desc="512 dense FP32 U diag(exp(-i/30)) V^T + noise, m, n ~ U[1000, 20000], "
                                 "rank ~ U[10, 100], k ~ U[16, 128], c=5",
                            l2="the batch's matrices are far larger than L2"))


class _Pool:
    """Resident inputs of the serving mix."""

    def __init__(self, cabs, torch, device, seed):
        from workloads import synth
        g = np.random.default_rng(seed)
        specs = synth.batched_specs(32, seed=seed + 1)
        self.dense = []
        for i, s in enumerate(specs):
            A, _, _, _ = synth.decaying_lowrank_device(s["m"], s["n"], rank=s["rank"], seed=seed + 31 * i,
                                                       device=device, noise_fp32=True)
            self.dense.append((cabs.dense_source(A), A))
        self.rbf = []
        for i, m in enumerate(sorted(g.integers(10000, 200001, size=6).tolist())):
            X, Y, sig = synth.rbf_mixture(m, m, d=16, seed=seed + 7 * i, sigma_pairs=1000)
            Xd, Yd = torch.from_numpy(X).to(device), torch.from_numpy(Y).to(device)
            self.rbf.append((cabs.rbf_source(Xd, Yd, sig), (Xd, Yd), m))
        A = synth.plain_lowrank(2000, 1500, seed=seed)
        Ad = torch.from_numpy(np.ascontiguousarray(A)).to(device)
        self.plain = (cabs.dense_source(Ad), Ad)


def serve_requests(cabs, pool, rate, seconds, seed, prec):
    """(arrival time, source, params) of a Poisson stream with the configured mix."""
    g = np.random.default_rng(seed)
    t, out, i = 0.0, [], 0
    while True:
        t += g.exponential(1.0 / rate)
        if t >= seconds:
            break
        u = g.random()
        if u < 0.50:
            s, A = pool.dense[g.integers(len(pool.dense))]
            m, n = A.shape
            k = int(g.integers(16, 129))
            p = cabs.make_params(m, n, min(k, m, n), iters=5, seed=int(seed + i), prec=prec, core="stabilized",
                                 trunc_rtol=min(k, m, n) * 2.0 ** -24,
                                 err_samples=0, err_seed=3)
        elif u < 0.95:
            s, _, m = pool.rbf[g.integers(len(pool.rbf))]
            k = int(g.integers(32, 257))
            p = cabs.make_params(m, m, k, iters=10, seed=int(seed + i), prec=prec, core="pinv", trunc_rtol=k * 2.0 ** -24,
                                 err_samples=100000, err_seed=3)
        else:
            s, _ = pool.plain
            p = cabs.make_params(2000, 1500, 20, iters=5, seed=int(seed + i), prec="fp64", core="pinv",
                                 err_samples=0, err_seed=3)
        out.append((t, s, p, "dense" if u < 0.50 else ("rbf" if u < 0.95 else "plain")))
        i += 1
    return out


def run_serve(args, cabs, torch, device, ctx, ClockSampler):
    rate, warm, seconds = 200.0, 5.0, args.serve_seconds
    pool = _Pool(cabs, torch, device, 1607)
    reqs = serve_requests(cabs, pool, rate, warm + seconds, 1607, args.prec)
    need = max(cabs.cabs_workspace_size(s, p) for _, s, p, _ in reqs)
    free, _ = torch.cuda.mem_get_info(device)
    arena = int(min(0.6 * free, max(16 * need, 8 << 30)))
    srv = cabs.Server(ctx, arena_bytes=arena, max_slots=8)
    lat, done_t, errs, pending, kinds, ivals = [], [], [], [], [], []
    sampler = ClockSampler(device.index or 0)
    l0 = cabs.cabs_launch_count()
    try:
        t0 = time.perf_counter()
        sampler.start()
        i = 0
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i][0] <= now:
                at, s, p, kind = reqs[i]
                pending.append((srv.submit(s, p), at, p, kind))
                i += 1
            still = []
            for tk, at, p, kind in pending:
                r = srv.poll(tk, timeout_ms=0)
                if r is None:
                    still.append((tk, at, p, kind))
                    continue
                res, ms = r
                if at >= warm:
                    lat.append(ms)
                    done_t.append(time.perf_counter() - t0)
                    errs.append(cabs.result_err(res, device))
                    kinds.append(kind)
                    ivals.append(srv.times(tk))
                srv.release(tk)
            pending = still
            if i < len(reqs):
                time.sleep(max(0.0, min(0.0005, reqs[i][0] - (time.perf_counter() - t0))))
            else:
                time.sleep(0.0002)
        clocks = sampler.stop()
    finally:
        srv.stop()
    launches = cabs.cabs_launch_count() - l0
    window = max(done_t) - warm if done_t else float("nan")
    per_kind = {}
    for kd in ("dense", "rbf", "plain"):
        e = [x for x, y in zip(errs, kinds) if y == kd]
        lk = [x for x, y in zip(lat, kinds) if y == kd]
        if e:
            per_kind[kd] = dict(requests=len(e), err_median=statistics.median(e), err_max=max(e),
                                lat_p50_ms=round(statistics.median(lk), 3), lat_p99_ms=round(_pct(lk, 0.99), 3))
    # device-time overlap: requests whose interval intersects another's
    iv = sorted(ivals)
    overlapped, reach = 0, -1.0
    flags = [False] * len(iv)
    for j, (a, b) in enumerate(iv):
        if a < reach:
            flags[j] = True
            flags[jmax] = True
        if b > reach:
            reach, jmax = b, j
    overlapped = sum(flags)

    # capacity: a fresh burst of the same request mix submitted all at once
    # (saturating arrivals), completions per second of wall time
    burst = [(s, p) for at, s, p, _ in reqs if at >= warm][:600]
    srv = cabs.Server(ctx, arena_bytes=arena, max_slots=8)
    try:
        t0 = time.perf_counter()
        tks = [srv.submit(s, p) for s, p in burst]
        for tk in tks:
            while srv.poll(tk, timeout_ms=100) is None:
                pass
            srv.release(tk)
        cap_s = time.perf_counter() - t0
    finally:
        srv.stop()

    # the plain FP32 form: the measured requests one at a time, back to back
    meas = [(s, p) for at, s, p, _ in reqs if at >= warm][:400]
    plain_ms = []
    qs = [cabs.make_params(p.m, p.n, p.k1, iters=p.iters, seed=p.seed,
                           prec="fp64" if p.prec == cabs.PRECS["fp64"] else "fp32", core=p.core,
                           trunc_rtol=p.trunc_rtol, err_samples=p.err_samples, err_seed=p.err_seed) for _, p in meas]
    ws = torch.empty(max(cabs.cabs_workspace_size(s, q) for (s, _), q in zip(meas, qs)) + 512, dtype=torch.uint8,
                     device=device)
    for (s, p), q in zip(meas, qs):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sk = cabs.cabs_sketch(ctx, s, q, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    mean_plain = statistics.mean(plain_ms)
    return dict(value=round(len(lat) / window, 4) if lat else None, steps=len(lat),
                ms_per_step=round(window * 1e3 / max(len(lat), 1), 4),
                latency_ms=dict(p50=round(statistics.median(lat), 3), p99=round(_pct(lat, 0.99), 3),
                                mean=round(statistics.mean(lat), 3)),
                rel_fro_error=dict(median=statistics.median(errs), max=max(errs)) if errs else None,
                per_kind=per_kind,
                capacity=dict(value=round(len(burst) / cap_s, 4), unit="sketches/s", requests=len(burst),
                              form="the measured mix submitted at once (saturating arrivals), 8 slots"),
                overlap=dict(requests=len(iv), overlapped=overlapped,
                             note="requests whose device-side interval (CUDA events on the slot stream) "
                                  "intersects another request's"),
                clocks=clocks, gpu_launches=int(launches),
                plain_fp32=dict(value=round(1e3 / mean_plain, 4), unit="sketches/s",
                                mean_service_ms=round(mean_plain, 3), sample=len(plain_ms),
                                form="the same requests one at a time, back to back, FP32 (plain requests FP64)"),
                config=dict(workload="serve", rate_per_s=rate, warmup_s=warm, measured_s=seconds,
                            requests=len(reqs), arena_gib=round(arena / 2**30, 1), max_slots=8, prec=args.prec,
                            mix="50% dense pool of 32 (batched distribution), 45% RBF m=n in [1e4, 2e5] "
                                "k in [32, 256], 5% plain FP64 2000x1500"))
