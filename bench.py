#!/usr/bin/env python
"""Benchmark: HGF multi-label aggregation + WTA on one GB300 (or N independent replicas).

One step = the whole hot path on one synthetic stereo workload already resident in device
memory: guidance precompute (polynomial guidance, moments, float64 covariance assembly and the
Prop. 1 inverse) followed by the fused aggregation of every label slice and WTA. The default
workload is the 450x375 stereo pair with 60 labels, degree-2 monomial guidance (n = 9), r = 9,
eps = 1e-4, float32 costs. The inputs (40.5 MB of costs) are smaller than L2, so a 256 MiB buffer
is written between timed steps (outside the timed events) to flush L2.

Metric: Mpixel*labels/s = H * W * L * steps / device time, summed over replicas.
Prints one JSON line (rank 0). --impl reference times the CPU oracle on a bounded crop instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel*labels/s HGF aggregate+WTA (n=9)"
UNIT = "Mpixel*labels/s"
WORKLOADS = {
    "quarter": dict(width=450, height=375, n_labels=60, degree=2, r=9, eps=1e-4, dtype="f32",
                    seed=2, name="stereo 450x375, L=60, RGB degree-2 monomials (n=9), r=9, "
                                 "eps=1e-4, float32 costs"),
    "small": dict(width=64, height=48, n_labels=16, degree=1, r=4, eps=1e-4, dtype="f32", seed=1,
                  name="stereo 64x48, L=16, RGB (n=3), r=4, eps=1e-4, float32 costs"),
    "large": dict(width=1400, height=1100, n_labels=256, degree=2, r=9, eps=1e-4, dtype="bf16",
                  seed=3, name="stereo 1400x1100, L=256, n=9, r=9, eps=1e-4, bf16 costs"),
    "deg3": dict(width=1280, height=960, n_labels=128, degree=3, r=4, eps=1e-4, dtype="bf16",
                 seed=19, name="stereo 1280x960, L=128, RGB degree-3 monomials (n=19), r=4, "
                               "eps=1e-4, bf16 costs"),
    "deg3small": dict(width=640, height=480, n_labels=64, degree=3, r=4, eps=1e-4, dtype="bf16",
                      seed=20, name="stereo 640x480, L=64, RGB degree-3 monomials (n=19), r=4, "
                                    "eps=1e-4, bf16 costs"),
}
FP32_LANES_PER_SM = 128                              # FP32 FMA lanes per SM (Blackwell)
FP64_PEAK_TFLOPS = 1.25                              # nominal GB300 FP64 rate


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 FMA peak from the queried SM count and an SM clock: SMs x 128 lanes x 2 flops."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def flops_per_unit(kernel: str, n: int) -> tuple[float, str] | None:
    """Algorithmic flops per unit (pixel*label for the aggregation kernels, pixel for the
    inverse) and the unit name."""
    if kernel == "k_fused":     # the whole per-label path: both box stages, cov, mat-vec,
        return 2 * n * n + 17 * n + 10, "px*label"   # offset, output and the WTA compare
    if kernel == "k_coef":      # n products, 5(n+1) box, 2n cov, 2n^2 mat-vec, 2n offset
        return 2 * n * n + 10 * n + 5, "px*label"
    if kernel == "k_apply":     # 5(n+1) box, 2n output, 1 compare
        return 7 * n + 6, "px*label"
    if kernel == "k_inverse":   # Prop. 1 recursion + assembly + read-off (float64)
        rec = sum(3 * k * k + 5 * k + 4 for k in range(n))
        return rec + 1.5 * n * (n + 1), "px"
    return None


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kernel` on
    `workload` from profiles/ncu_traffic.md, or None when there is no capture or the kernel's
    source file has changed since (the capture records a sha256 prefix of that file)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) == 5 and cells[0] == kernel and cells[1] == workload:
            src = os.path.join(ROOT, cells[3])
            if not os.path.exists(src):
                return None
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            return float(cells[2]) if sha == cells[4] else None
    return None


def world_max(x: float, dist, device) -> float:
    """Maximum of a per-rank float over all ranks (device: where the collective's tensor lives:
    CUDA for NCCL, CPU for gloo)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, world: int, t_max_s: float) -> float:
    """Whole-job throughput in Mpixel*labels/s: every replica processes the same units; the job
    takes as long as the slowest rank."""
    return world * units_per_rank / t_max_s / 1e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["fused", "plain", "reference"], default="fused")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="quarter")
    ap.add_argument("--kernel", type=int, choices=[0, 1, 2], default=0,
                    help="fused path: 0 automatic, 1 single-pass kernel, 2 two kernels")
    ap.add_argument("--labels-per-pass", type=int, choices=[0, 1, 2, 4, 8], default=0,
                    help="two-kernel path: labels per pass of the coefficient kernel (0 auto)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--inv-precision", choices=["f64", "df64", "f32"], default="f64",
                    help="arithmetic of the covariance assembly + inverse")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the warm, plain-form, single-pass and served legs of the line")
    ap.add_argument("--serve-rate", type=float, default=20.0,
                    help="requests per second of the default line's short served leg")
    ap.add_argument("--cpu-crop", type=int, nargs=2, default=None,
                    help="width height of the centred crop the CPU baseline runs on (default: "
                         "the largest whose two repetitions take about 15 s)")
    ap.add_argument("--serve", action="store_true",
                    help="open-loop serving run (Poisson arrivals) instead of the step benchmark")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean requests per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--warm", type=float, default=2.0, help="serving: seconds before measuring")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--batch", action="store_true",
                    help="32 mixed-size stereo pairs as one batch, one captured graph per step")
    ap.add_argument("--streams", type=int, default=8, help="batch: internal streams")
    ap.add_argument("--inverse", action="store_true",
                    help="batched-inverse microbenchmark: Prop. 1 vs per-matrix Cholesky")
    ap.add_argument("--count", type=int, default=1_000_000, help="inverse: matrices per batch")
    ap.add_argument("--table3", action="store_true",
                    help="the paper's Table 3 shape: one gray slice, paper form, n = 3..9 powers")
    return ap.parse_args()


# Table 3 of the paper (GTX 960, ArrayFire; ms per filtered slice), context only
PAPER_TABLE3_MS = {250: (3.9, 10.7, 39.9, 110.2), 500: (3.7, 11.1, 40.1, 112.4),
                   1000: (4.1, 10.9, 41.3, 115.9), 2000: (4.3, 11.2, 42.7, 121.8)}


def table3_arm(args):
    """The paper's Table 3 workload shape: a gray image of 250^2 .. 2000^2 filtering one slice
    (itself) with the paper's own form (G_0 = 1, uncentred sums, lambda = 0.05 in sum units,
    r = 7) and power guidance I, I^2, .., I^n for n = 3, 5, 7, 9. One step = guidance precompute
    + aggregation of the slice with the filtered output written. Median of `steps` CUDA-event
    timed steps after warm-up, L2 flushed between steps."""
    import numpy as np
    import torch
    from paper_1803_00005_gb300 import build, hgf, synth
    build.build()
    torch.cuda.set_device(0)
    ctx = hgf.hgf_create(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    reps = max(5, min(args.steps, 50))
    table = []
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = hgf.hgf_launch_count(ctx)
    for size in (250, 500, 1000, 2000):
        left, _, _ = synth.stereo_pair(size, size, 16, 300 + size)
        gray = left.mean(axis=0, keepdims=True).astype(np.float32)
        img = torch.from_numpy(gray).cuda()
        cost = img.clone()                                  # the slice: the image itself
        out = torch.empty_like(cost)
        for j, n in enumerate((3, 5, 7, 9)):
            g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=n, r=7, eps=0.05,
                                                          basis="powers", form="paper"))
            for _ in range(max(3, args.warmup)):
                hgf.hgf_guidance_update(ctx, g, img)
                hgf.hgf_aggregate(ctx, g, cost, filtered=out)
            ms = []
            for i in range(reps):
                flush.fill_(i & 0xff)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                hgf.hgf_guidance_update(ctx, g, img)
                hgf.hgf_aggregate(ctx, g, cost, filtered=out)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            hgf.hgf_guidance_release(g)
            t = statistics.median(ms)
            table.append(dict(size=size, n=n, ms=t, mpx_per_s=size * size / t / 1e3,
                              paper_gtx960_ms=PAPER_TABLE3_MS[size][j]))
    clk = clocks.stop()
    launches = hgf.hgf_launch_count(ctx) - launches0
    hgf.hgf_destroy(ctx)
    key = next(r for r in table if r["size"] == 1000 and r["n"] == 9)
    line = dict(metric="ms per filtered gray slice, paper form, n=9 powers, 1000x1000",
                value=key["ms"], unit="ms", n_gpus=1, steps=reps, warmup=max(3, args.warmup),
                ms_per_step=key["ms"], higher_is_better=False, scaling="weak", vs_baseline=None,
                dtype="f32 (f64 inverse)", data="synthetic", impl="table3",
                config=dict(workload="gray 250^2..2000^2, one slice, paper form, lambda=0.05, "
                                     "r=7, powers n=3,5,7,9 (the shape of the paper's Table 3)",
                            l2="256 MiB flush between steps",
                            step="guidance precompute + aggregate (filtered output)"),
                table=table, gpu_launches=launches, clocks=clk,
                note="paper_gtx960_ms: the paper's Table 3 (GTX 960), context only")
    print(json.dumps(line), flush=True)


def inverse_arm(args):
    """Batched (lambda E + S_i)^-1 of 10^6 seeded Gram matrices (25 samples of U[0,1]^n each,
    lambda = 0.05), n = 3, 6, 9, 19: Prop. 1's recursion against per-matrix Cholesky, float64 and
    float32 arithmetic, one thread per matrix (Sec. 3, Fig. 1b). A 256 MiB buffer is written
    between timed launches to flush L2. value = Prop. 1, float64, n = 9, matrices/s."""
    import torch
    from paper_1803_00005_gb300 import build, hgf, synth
    build.build()
    torch.cuda.set_device(0)
    ctx = hgf.hgf_create(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    reps = max(3, min(args.steps, 20))
    table = []
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = hgf.hgf_launch_count(ctx)
    for n in (3, 6, 9, 19):
        S = synth.pack_upper(synth.gram_batch_torch(args.count, n, seed=11 + n))
        out = torch.empty_like(S)
        for method in ("prop1", "cholesky"):
            for prec in ("f64", "df64", "f32"):
                for _ in range(max(3, args.warmup)):
                    hgf.hgf_batched_inverse(ctx, S, n, 0.05, method, prec, out)
                ms = []
                for i in range(reps):
                    flush.fill_(i & 0xff)
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    hgf.hgf_batched_inverse(ctx, S, n, 0.05, method, prec, out)
                    b.record(stream)
                    b.synchronize()
                    ms.append(a.elapsed_time(b))
                t = statistics.median(ms) / 1e3
                P = n * (n + 1) // 2
                table.append(dict(n=n, method=method, precision=prec,
                                  matrices_per_s=args.count / t, ms=1e3 * t,
                                  gbs=2 * P * 8 * args.count / t / 1e9))
        del S, out
    clk = clocks.stop()
    launches = hgf.hgf_launch_count(ctx) - launches0
    hgf.hgf_destroy(ctx)
    key = next(r for r in table if r["n"] == 9 and r["method"] == "prop1" and
               r["precision"] == "f64")
    ratio = {f"n={n} {prec}": next(r["ms"] for r in table if r["n"] == n and
                                   r["method"] == "cholesky" and r["precision"] == prec) /
             next(r["ms"] for r in table if r["n"] == n and r["method"] == "prop1" and
                  r["precision"] == prec)
             for n in (3, 6, 9, 19) for prec in ("f64", "df64", "f32")}
    line = dict(metric="matrices/s, batched (lambda E + S)^-1, Prop. 1, n=9, float64",
                value=key["matrices_per_s"], unit="matrices/s", n_gpus=1, steps=reps,
                warmup=max(3, args.warmup), ms_per_step=key["ms"], higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="inverse",
                config=dict(workload=f"{args.count} Gram matrices of 25 U[0,1]^n samples, "
                                     "lambda=0.05, packed float64 in and out",
                            l2="256 MiB flush between launches"),
                table=table, cholesky_over_prop1_time=ratio, gpu_launches=launches,
                clocks=clk)
    print(json.dumps(line), flush=True)


def batch_arm(args):
    """Mixed-size batch (synth.batched_cases: 8 each of 320x240, 640x480, 1024x768, 1280x960;
    L in {32, 64, 128, 192}; degree 1 or 2; r in {4, 9}; float32 costs built on the device).
    One step = one launch of the captured graph holding every job's precompute, aggregation and
    WTA. value: the single-pass kernel's persistent launch over all 32 jobs (the graph holds the
    32 precomputes on the internal streams, one persistent aggregation launch and the WTA
    unpacking); streams_graph: the same batch with each job's two-kernel aggregation on the
    internal streams. Inputs total > L2 (no flush needed)."""
    import numpy as np
    import torch
    from paper_1803_00005_gb300 import build, hgf, synth
    build.build()
    torch.cuda.set_device(0)
    specs = synth.batched_cases(32, 400)
    ctx = hgf.hgf_create(0)
    jobs, keep, units, in_bytes = [], [], 0, 0
    for sp in specs:
        left, right, _ = synth.stereo_pair(sp["width"], sp["height"], sp["n_labels"], sp["seed"])
        img = torch.from_numpy(left.astype(np.float32)).cuda()
        cost = synth.cost_volume_torch(left, right, sp["n_labels"], "f32")
        lab = torch.empty((sp["height"], sp["width"]), dtype=torch.int32, device="cuda")
        p = hgf.make_params(degree=sp["degree"], r=sp["r"], eps=sp["eps"])
        jobs.append(hgf.make_job(img, cost, p, labels=lab))
        keep.append((img, cost, lab))
        units += sp["width"] * sp["height"] * sp["n_labels"]
        in_bytes += cost.numel() * 4 + img.numel() * 4
    stream = torch.cuda.current_stream()
    steps = max(1, min(args.steps, 20))

    def time_graph(kernel):
        hgf.hgf_set_tuning(ctx, kernel=kernel)
        batch = hgf.hgf_batch_create(ctx, jobs, streams=args.streams)
        for _ in range(max(1, args.warmup)):
            hgf.hgf_batch_launch_graph(ctx, batch)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for i in range(steps):
            hgf.hgf_batch_launch_graph(ctx, batch)
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        hgf.hgf_batch_destroy(batch)
        return ev[0].elapsed_time(ev[-1]) / 1e3

    clocks = ClockSampler(0)
    clocks.start()
    t_joint = time_graph(1)
    t_streams = time_graph(0)
    clk = clocks.stop()
    hgf.hgf_destroy(ctx)
    line = dict(metric="Mpixel*labels/s HGF aggregate+WTA, mixed batch",
                value=units * steps / t_joint / 1e6,
                unit=UNIT, n_gpus=1, steps=steps, warmup=args.warmup,
                ms_per_step=1e3 * t_joint / steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32 (f64 inverse)", data="synthetic", impl="batch",
                config=dict(workload="32 stereo pairs, 8 each of 320x240/640x480/1024x768/"
                                     "1280x960, L in {32,64,128,192}, degree 1 or 2, r in {4,9}, "
                                     "float32 costs; one captured graph per step: the precomputes "
                                     f"on {args.streams} streams, one persistent single-pass "
                                     "aggregation launch over all jobs, WTA unpacking",
                            l2=f"inputs {in_bytes / 2**20:.0f} MiB > L2",
                            units_per_step=units),
                streams_graph=dict(value=units * steps / t_streams / 1e6, unit=UNIT,
                                   ms_per_step=1e3 * t_streams / steps,
                                   note=f"every job's precompute and two-kernel aggregation on "
                                        f"{args.streams} internal streams, one captured graph"),
                clocks=clk)
    print(json.dumps(line), flush=True)


def run_serving(rate, duration, warm, slots, device=0):
    """Open-loop serving: requests arrive at Poisson times (synth.serving_requests: sizes
    640x480 .. 1920x1080, L 64..256, degree 1..3, r in {4, 9}, bf16 costs, 30% reuse an earlier
    guidance) and are submitted to hgf_serve at their arrival time; latency counts from the
    scheduled arrival. Inputs come from a pool of device-resident stereo pairs per size (costs
    built on the device before the clock starts). Returns hgf_serve_stats after the run (the
    statistics are reset once the warm-up's arrivals are submitted)."""
    import numpy as np
    import torch
    from paper_1803_00005_gb300 import hgf, synth
    n_req = int(rate * (duration + warm)) + 1
    reqs = synth.serving_requests(n_req, rate_hz=rate, seed=5)
    pool = {}
    for sp in reqs:
        key = (sp["width"], sp["height"])
        if key not in pool:
            left, right, _ = synth.stereo_pair(sp["width"], sp["height"], 256, 5000 + len(pool))
            pool[key] = dict(img=torch.from_numpy(left.astype(np.float32)).cuda(),
                             cost=synth.cost_volume_torch(left, right, 256, "bf16"),
                             labels=torch.empty((sp["height"], sp["width"]), dtype=torch.int32,
                                                device="cuda"))
    torch.cuda.synchronize()
    srv = hgf.hgf_serve_create(device, budget_bytes=120 << 30, slots=slots, max_queue=4096,
                               max_pixels=1920 * 1080, max_n=19)
    t0 = time.perf_counter() + 0.5
    ids, measured = [], []
    warm_end = None
    for i, sp in enumerate(reqs):
        p = pool[(sp["width"], sp["height"])]
        params = hgf.make_params(degree=sp["degree"], r=sp["r"], eps=sp["eps"])
        cost = p["cost"][:sp["n_labels"]]
        req = hgf.make_request(sp["guidance_key"], p["img"], cost, params, p["labels"])
        now = time.perf_counter()
        wait = t0 + sp["arrival_s"] - now
        if wait > 0:
            time.sleep(wait)
        if warm_end is None and sp["arrival_s"] >= warm:
            hgf.hgf_serve_stats(srv, reset=True)
            warm_end = i
        st, rid = hgf.hgf_serve_submit(srv, req)
        ids.append((st, rid))
    for st, rid in ids:
        if st == hgf.HGF_OK:
            hgf.hgf_serve_wait(srv, rid, 600000)
    stats = hgf.hgf_serve_stats(srv)
    hgf.hgf_serve_destroy(srv)
    del pool
    torch.cuda.empty_cache()
    return stats


def serve_arm(args):
    """The serving run of run_serving at --rate for --duration seconds after --warm seconds."""
    import torch
    from paper_1803_00005_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stats = run_serving(args.rate, args.duration, args.warm, args.slots)
    line = dict(metric="served HGF aggregate+WTA: p50/p99 latency and throughput",
                value=stats["mpixel_labels_per_s"], unit=UNIT, n_gpus=1,
                higher_is_better=True, impl="serve", data="synthetic",
                config=dict(workload=f"Poisson {args.rate:g} req/s for {args.duration:g} s after "
                                     f"{args.warm:g} s warm-up; 640x480..1920x1080, L 64..256, "
                                     f"n in {{3, 9, 19}}, r in {{4, 9}}, bf16 costs, 30% guidance "
                                     f"reuse, 120 GiB budget, {args.slots} slots"),
                serve=stats)
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ CPU oracle arm
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth
w = {w!r}
case = synth.make_case(w["width"], w["height"], w["n_labels"], w["seed"], w["dtype"])
cw, ch = {crop!r}
H, W = w["height"], w["width"]
y0, x0 = (H - ch) // 2, (W - cw) // 2
I = case.guidance[:, y0:y0 + ch, x0:x0 + cw]
P = synth.from_dtype(case.cost[:, y0:y0 + ch, x0:x0 + cw], w["dtype"])
times = []
for rep in range({reps}):
    t = time.perf_counter()
    q = O.centred_filter(I, P, w["r"], w["eps"], w["degree"])
    labels = O.wta(q)[0]
    times.append(time.perf_counter() - t)
print(json.dumps(dict(times=times, units=cw * ch * P.shape[0])))
"""


ORACLE_POOL_SNIPPET = r"""
import json, os, sys, time, multiprocessing as mp
sys.path.insert(0, {root!r})

def work(args):
    import numpy as np
    from oracle import hgf_oracle as O
    I, P, w = args
    q = O.centred_filter(I, P, w["r"], w["eps"], w["degree"])
    return np.argmin(q, axis=0)

if __name__ == "__main__":
    import numpy as np
    from paper_1803_00005_gb300 import synth
    w = {w!r}
    case = synth.make_case(w["width"], w["height"], w["n_labels"], w["seed"], w["dtype"])
    cw, ch = {crop!r}
    H, W = w["height"], w["width"]
    y0, x0 = (H - ch) // 2, (W - cw) // 2
    I = case.guidance[:, y0:y0 + ch, x0:x0 + cw]
    P = synth.from_dtype(case.cost[:, y0:y0 + ch, x0:x0 + cw], w["dtype"])
    cores = len(os.sched_getaffinity(0))
    chunks = [c for c in np.array_split(np.arange(P.shape[0]), cores) if len(c)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(chunks)) as pool:
        pool.map(work, [(I[:, :4, :4], P[c][:, :4, :4], w) for c in chunks])   # start-up
        times = []
        for rep in range({reps}):
            t = time.perf_counter()
            pool.map(work, [(I, P[c], w) for c in chunks])
            times.append(time.perf_counter() - t)
    print(json.dumps(dict(times=times, units=cw * ch * P.shape[0], cores=len(chunks))))
"""


def run_oracle_pool(w, crop, reps):
    """Times the CPU oracle with the labels split over every host core (one spawned process per
    core, each with one BLAS/OpenMP thread; each process recomputes the guidance part)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_POOL_SNIPPET.format(root=ROOT, w=w, crop=tuple(crop), reps=reps)
    with tempfile.NamedTemporaryFile("w", suffix=".py", delete=False) as f:
        f.write(code)
        path = f.name
    try:
        out = subprocess.run([sys.executable, path], capture_output=True, text=True, env=env,
                             timeout=1800)
    finally:
        os.unlink(path)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle(w, crop, reps):
    """Times the CPU oracle (float64, single thread) on a centred crop with all labels, in a
    fresh interpreter (no GPU state, BLAS/OpenMP pinned to one thread)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, w=w, crop=tuple(crop), reps=reps)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# The oracle's measured rate on the GPU machine's host (one core, 450x375 / L = 60 / n = 9), used only to
# size the reference arm's sample so that its run stays within a few minutes.
PROFILE_EVERY = 10  # timed steps per profiled step (per-kernel events)
ORACLE_MPLS_ESTIMATE = 1.05
REFERENCE_BUDGET_S = 150.0


CPU_SAMPLE_S = 15.0  # target CPU time of the default line's cpu_baseline (two repetitions)


def cpu_sample_crop(w):
    """The whole workload, or the largest centred crop (same aspect), whose two oracle repetitions
    take about CPU_SAMPLE_S at the oracle's measured rate, scaled from n = 9 by the flops per
    px*label (2n^2 + 17n + 10) of the workload's degree."""
    n = {1: 3, 2: 9, 3: 19}.get(w["degree"], 9)
    rate = ORACLE_MPLS_ESTIMATE * 325.0 / (2 * n * n + 17 * n + 10)
    full = w["width"] * w["height"] * w["n_labels"]
    fit = CPU_SAMPLE_S * rate * 1e6 / 2
    if full <= fit:
        return (w["width"], w["height"])
    s = (fit / full) ** 0.5
    return (max(8, int(w["width"] * s)), max(8, int(w["height"] * s)))


def reference_crop(w, steps_total):
    """The whole image when (warm-up + timed) oracle steps on it fit the time budget at the
    estimated rate, else the largest centred crop (same aspect) that does."""
    full = w["width"] * w["height"] * w["n_labels"]
    fit = REFERENCE_BUDGET_S * ORACLE_MPLS_ESTIMATE * 1e6 / max(1, steps_total)
    if full <= fit:
        return (w["width"], w["height"])
    s = (fit / full) ** 0.5
    return (max(8, int(w["width"] * s)), max(8, int(w["height"] * s)))


def reference_arm(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    crop = reference_crop(w, args.warmup + args.steps)
    res = run_oracle(w, crop, args.warmup + args.steps)
    t = res["times"][args.warmup:]
    total = sum(t)
    value = res["units"] * len(t) / total / 1e6
    whole = crop == (w["width"], w["height"])
    sample = ((f"the whole {w['width']}x{w['height']} workload" if whole else
               f"centred {crop[0]}x{crop[1]} crop of the {w['width']}x{w['height']} workload") +
              f", all {w['n_labels']} labels, prepare + aggregate + WTA per step, float64 numpy, "
              f"one thread")
    config = dict(workload=w["name"], parallelism="replicas x1",
                  step="guidance precompute + aggregate + WTA", l2="n/a (CPU oracle)")
    if not whole:
        config["sample"] = sample
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * total / len(t), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference", config=config,
                cpu_baseline=dict(value=value, unit=UNIT, cores=1, kind="oracle", sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))


# ---------------------------------------------------------------------------------- GPU arm
def timed_leg(step, steps, flush, stream):
    """Per-step device times (ms) of `steps` calls of step(), each bracketed by CUDA events on
    `stream`, with the L2 flush written between steps (outside the events)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_((i + 3) & 0xff)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def main():
    args = parse()
    w = WORKLOADS[args.workload]
    if args.serve:
        return serve_arm(args)
    if args.batch:
        return batch_arm(args)
    if args.inverse:
        return inverse_arm(args)
    if args.table3:
        return table3_arm(args)
    if args.impl == "reference":
        return reference_arm(args, w)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        crop = ((min(args.cpu_crop[0], w["width"]), min(args.cpu_crop[1], w["height"]))
                if args.cpu_crop else cpu_sample_crop(w))
        res = run_oracle(w, crop, 2)            # before any GPU work in this process
        tot = sum(res["times"])
        cpu = dict(value=res["units"] * len(res["times"]) / tot / 1e6, unit=UNIT, cores=1,
                   kind="oracle",
                   sample=(f"the whole {w['width']}x{w['height']} workload"
                           if crop == (w["width"], w["height"]) else
                           f"centred {crop[0]}x{crop[1]} crop") +
                          f", all {w['n_labels']} labels, prepare + aggregate + WTA, 2 repetitions "
                          f"({tot:.1f} s), float64 numpy, one thread")
        try:
            resp = run_oracle_pool(w, crop, 2)
            tp = sum(resp["times"])
            cpu_all = dict(value=resp["units"] * len(resp["times"]) / tp / 1e6, unit=UNIT,
                           cores=resp["cores"], kind="oracle",
                           sample=f"same sample, labels split over {resp['cores']} spawned "
                                  f"processes (one thread each), 2 repetitions ({tp:.1f} s)")
        except (RuntimeError, subprocess.TimeoutExpired, OSError) as exc:
            cpu_all = dict(value=None, error=str(exc)[-300:])

    import numpy as np
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    from paper_1803_00005_gb300 import build, hgf, synth
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    case = synth.make_case(w["width"], w["height"], w["n_labels"], w["seed"], w["dtype"])
    L, H, W = case.cost.shape
    n = hgf.hgf_num_channels(3, w["degree"])
    img = torch.from_numpy(case.guidance).to(dev)
    if w["dtype"] == "bf16":
        cost = torch.from_numpy(case.cost.view(np.int16)).to(dev).view(torch.bfloat16)
    else:
        cost = torch.from_numpy(case.cost).to(dev)
    labels = torch.empty((H, W), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    ctx = hgf.hgf_create(local_rank)
    params = hgf.make_params(degree=w["degree"], r=w["r"], eps=w["eps"],
                             inv_precision=args.inv_precision)
    g = hgf.hgf_prepare(ctx, img, params)
    agg = hgf.hgf_aggregate_plain if args.impl == "plain" else hgf.hgf_aggregate
    if args.kernel or args.labels_per_pass:
        hgf.hgf_set_tuning(ctx, kernel=args.kernel, labels_per_pass=args.labels_per_pass)

    def step():
        # one frame: guidance precompute + aggregation + WTA (hgf_filter: both in one call)
        if args.impl == "plain":
            hgf.hgf_guidance_update(ctx, g, img)
            agg(ctx, g, cost, labels=labels)
        else:
            hgf.hgf_filter(ctx, g, img, cost, labels=labels)

    for i in range(args.warmup):
        flush.fill_(i & 0xff)
        step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = hgf.hgf_launch_count(ctx)
    # per-kernel CUDA events (the library's profiler) on every PROFILE_EVERY-th timed step: the
    # event pairs around each launch cost about 3 % of a step, so the other steps run without them
    profiled = [i for i in range(args.steps) if i % PROFILE_EVERY == 0]
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_((i + 7) & 0xff)           # L2 flush, outside the step's events
        if i % PROFILE_EVERY == 0:
            hgf.hgf_profile_enable(ctx, True)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
        if i % PROFILE_EVERY == 0:
            hgf.hgf_profile_enable(ctx, False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = hgf.hgf_launch_count(ctx) - launches0
    main_path = {1: "single pass (k_fused)", 2: "two kernels (k_coef + k_apply)",
                 3: "plain form"}.get(hgf.hgf_last_plan(ctx)["path"], "?")
    prof = hgf.hgf_profile_report(ctx)
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_dev = sum(step_ms) / 1e3
    t_max = world_max(t_dev, dist, dev) if world > 1 else t_dev
    units = H * W * L * args.steps
    value = whole_job_value(units, world, t_max)

    # roofline of the dominant kernel (largest share of the profiled time); the FP32 peak from
    # the device's SM count and the SM clock sampled during the timed region
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    fp32_peak = fp32_peak_tflops(sm_count, sm_mhz)
    kernels = {k: dict(launches=v["launches"], ms_per_step=v["ms"] / len(profiled),
                       profiled_steps=len(profiled))
               for k, v in prof.items()}
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])[0] if prof else None
    roof = None
    if dom is not None:
        fu = flops_per_unit(dom, n)
        avg_s = prof[dom]["ms"] / prof[dom]["launches"] / 1e3
        if fu is not None:
            per_unit, uname = fu
            launches_per_step = prof[dom]["launches"] / len(profiled)
            units_per_launch = (H * W * L if uname == "px*label" else H * W) / launches_per_step
            achieved = per_unit * units_per_launch / avg_s / 1e12
            peak = FP64_PEAK_TFLOPS if dom == "k_inverse" else fp32_peak
            roof = dict(bound="alu", kernel=dom, achieved=achieved, peak=peak, unit="TFLOP/s",
                        frac=achieved / peak, traffic=profiled_traffic(dom, args.workload),
                        model=f"{per_unit:.0f} flops per {uname}",
                        peak_note=("nominal float64 rate" if dom == "k_inverse" else
                                   f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                                   f"x {sm_mhz:.0f} MHz (median SM clock sampled under load)"))

    # further legs on the same inputs (rank 0 of a single-GPU run): the aggregation alone with the
    # guidance resident (warm; the precompute is timed separately per the metric's definition),
    # the plain form's cold step, the single-pass kernel (cold and warm), a short served run
    extra = {}
    if rank == 0 and world == 1 and args.impl == "fused" and not args.no_extra:
        flushes = flush
        warm_ms = timed_leg(lambda: agg(ctx, g, cost, labels=labels), args.steps, flushes, stream)
        prep_ms = timed_leg(lambda: hgf.hgf_guidance_update(ctx, g, img), args.steps, flushes,
                            stream)
        extra["warm"] = dict(value=H * W * L * len(warm_ms) / (sum(warm_ms) / 1e3) / 1e6,
                             unit=UNIT, ms_per_step=statistics.mean(warm_ms),
                             precompute_ms=statistics.mean(prep_ms),
                             note="aggregate + WTA with the guidance moments and inverse "
                                  "resident; precompute_ms: the guidance precompute alone")
        np_steps = max(3, min(args.steps, 30))

        def plain_step():
            hgf.hgf_guidance_update(ctx, g, img)
            hgf.hgf_aggregate_plain(ctx, g, cost, labels=labels)
        plain_step()
        plain_ms = timed_leg(plain_step, np_steps, flushes, stream)
        plain_value = H * W * L * len(plain_ms) / (sum(plain_ms) / 1e3) / 1e6
        extra["plain"] = dict(value=plain_value, unit=UNIT, ms_per_step=statistics.mean(plain_ms),
                              steps=np_steps, fused_over_plain=value / plain_value,
                              note="plain FP32 single-request GPU form: one kernel per step "
                                   "(products, row sums, column sums, coefficients, output, WTA),"
                                   " same step (precompute + aggregate + WTA)")
        saved_kernel = args.kernel
        notes = {1: "hgf_tuning.kernel = 1: k_fused, slice moments to WTA in one persistent pass",
                 2: "hgf_tuning.kernel = 2: k_coef (coefficients to a workspace) + k_apply "
                    "(their box filter, output, WTA)"}
        for kern, key in ((1, "single_pass"), (2, "two_kernel")):
            hgf.hgf_set_tuning(ctx, kernel=kern)
            step()
            sp_ms = timed_leg(step, args.steps, flushes, stream)
            spw_ms = timed_leg(lambda: agg(ctx, g, cost, labels=labels), args.steps, flushes,
                               stream)
            extra[key] = dict(
                value=H * W * L * len(sp_ms) / (sum(sp_ms) / 1e3) / 1e6, unit=UNIT,
                ms_per_step=statistics.mean(sp_ms),
                warm_value=H * W * L * len(spw_ms) / (sum(spw_ms) / 1e3) / 1e6,
                note=notes[kern] + " (same step; warm_value: aggregation alone)")
        hgf.hgf_set_tuning(ctx, kernel=saved_kernel)

    # whole-step HBM fraction from the algorithmic bytes per px*label: the cost read once plus
    # the guidance image, inverse record and label write per pixel (amortised over L)
    sc = {"f32": 4, "bf16": 2, "f16": 2}[w["dtype"]]
    bytes_per_unit = sc + (12 + 4 * (n * (n + 1) // 2 + n) + 4) / L
    hbm_peak = None
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, ValueError, KeyError):
        pass
    hbm = None
    if hbm_peak:
        gbs = bytes_per_unit * H * W * L * args.steps / t_max / 1e9 * world
        hbm = dict(algorithmic_gbs=gbs, peak_gbs=hbm_peak, frac=gbs / hbm_peak,
                   bytes_per_px_label=bytes_per_unit, peak_note="measured (MEASURED_PEAKS.json)")

    e2e = None
    if not args.no_e2e:
        pin_img = torch.from_numpy(case.guidance).pin_memory()
        raw = case.cost.view(np.int16) if w["dtype"] == "bf16" else case.cost
        pin_cost = torch.from_numpy(np.ascontiguousarray(raw)).pin_memory()
        pin_lab = torch.empty((H, W), dtype=torch.int32).pin_memory()
        hctx = hgf.hgf_create(local_rank)
        hgf.hgf_filter_host(hctx, pin_img.numpy(), pin_cost.numpy(), w["dtype"], params,
                            pin_lab.numpy())
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hgf.hgf_filter_host(hctx, pin_img.numpy(), pin_cost.numpy(), w["dtype"], params,
                                pin_lab.numpy())
        te = time.perf_counter() - t0
        hgf.hgf_destroy(hctx)
        if world > 1:
            te = world_max(te, dist, dev)
        e2e = dict(value=whole_job_value(units, world, te), unit=UNIT,
                   h2d_bytes_per_step=int(pin_img.numel() * 4 + pin_cost.numel() *
                                          pin_cost.element_size()),
                   d2h_bytes_per_step=int(H * W * 4))

    # end to end from the stereo pair itself through hgf_stereo_host: both views uploaded from
    # pinned host memory, the cost computed inside the coefficient kernel, labels read back;
    # `stereo_pipeline` adds the right view's aggregation and the left-right refinement
    e2e_stereo = stereo_pipeline = None
    if not args.no_e2e and args.impl == "fused":
        left, right, _ = synth.stereo_pair(W, H, L, w["seed"])
        pin_l = torch.from_numpy(left.astype(np.float32)).pin_memory()
        pin_r = torch.from_numpy(right.astype(np.float32)).pin_memory()
        pin_d = torch.empty((H, W), dtype=torch.int32).pin_memory()
        sctx = hgf.hgf_create(local_rank)

        def run_pipeline(refine, steps):
            for _ in range(3):
                hgf.hgf_stereo_host(sctx, pin_l.numpy(), pin_r.numpy(), L, params, refine=refine,
                                    out=pin_d.numpy())
            t0 = time.perf_counter()
            for _ in range(steps):
                hgf.hgf_stereo_host(sctx, pin_l.numpy(), pin_r.numpy(), L, params, refine=refine,
                                    out=pin_d.numpy())
            ts = time.perf_counter() - t0
            return world_max(ts, dist, dev) if world > 1 else ts

        ts = run_pipeline(False, args.steps)
        e2e_stereo = dict(value=whole_job_value(units, world, ts), unit=UNIT,
                          h2d_bytes_per_step=int(2 * pin_l.numel() * 4),
                          d2h_bytes_per_step=int(H * W * 4),
                          note="hgf_stereo_host: stereo pair in, disparity out; cost computed "
                               "on the device inside the coefficient kernel")
        nref = max(3, args.steps // 4)
        tr = run_pipeline(True, nref)
        stereo_pipeline = dict(ms_per_frame=1e3 * tr / nref,
                               note="hgf_stereo_host with refinement: cost, aggregation and WTA "
                                    "for both views, left-right check, hole filling; from host "
                                    "views to host disparity")
        hgf.hgf_destroy(sctx)

    hgf.hgf_guidance_release(g)
    hgf.hgf_destroy(ctx)
    if rank == 0 and world == 1 and args.impl == "fused" and not args.no_extra:
        del flush
        torch.cuda.empty_cache()
        st = run_serving(args.serve_rate, 3.0, 1.0, args.slots, device=local_rank)
        extra["served"] = dict(
            value=st["mpixel_labels_per_s"], unit=UNIT, p50_ms=st["p50_ms"], p99_ms=st["p99_ms"],
            completed=st["completed"], rate_hz=args.serve_rate,
            note=f"hgf_serve: Poisson {args.serve_rate:g} req/s for 3 s after 1 s warm-up; "
                 "640x480..1920x1080, L 64..256, n in {3, 9, 19}, r in {4, 9}, bf16 costs, 30% "
                 f"guidance reuse, 120 GiB budget, {args.slots} slots; latency from the "
                 "scheduled arrival")
    if rank == 0:
        metric = METRIC if n == 9 else METRIC.replace("(n=9)", f"(n={n})")
        line = dict(metric=metric, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=1e3 * t_max / args.steps,
                    higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype=f"f32 ({args.inv_precision} inverse)", data="synthetic",
                    impl=args.impl,
                    config=dict(workload=w["name"], parallelism=f"replicas x{world}",
                                l2="256 MiB buffer written between timed steps",
                                step="guidance precompute + aggregate + WTA"
                                     + ("" if args.impl == "plain" else " (one hgf_filter call)"),
                                path=main_path),
                    roofline=roof, hbm=hbm, cpu_baseline=cpu,
                    cpu_baseline_all_cores=cpu_all, e2e=e2e, e2e_stereo=e2e_stereo,
                    stereo_pipeline=stereo_pipeline,
                    gpu_launches=int(launches),
                    clocks=clk, kernels=kernels, wall_s=wall,
                    step_ms=dict(min=min(step_ms), median=statistics.median(step_ms)),
                    **extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
