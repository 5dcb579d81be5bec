"""Benchmark: batched complex64 FFTs on GB300 through the library's C ABI.

One step = one pass of the power-of-two sweep: for n = 2^4 .. 2^24 a batch of
2^26 / n contiguous transforms (512 MiB in, 512 MiB out), forward and
backward, plus a rank-2 4096 x 4096 transform and a single n = 2^24 transform,
forward and backward.  Inputs are seeded uniform[-1, 1) complex64, resident in
HBM and larger than L2 (no flush needed).

Prints one JSON line.  ``value`` is GFLOP/s under the 5 N log2 N convention,
summed over every transform of the step, divided by the device time of the
step (CUDA events, max over ranks); ``e2e`` repeats the measurement through
the same C ABI with host buffers (pinned host -> device copy of each input and
device -> host copy of each output inside the timed region).

``--impl reference`` times the FP64 CPU oracle (the only reference this
project has) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fft_inputs  # noqa: E402

METRIC = "C2C FFT GFLOP/s (5n log2 n) + HBM roofline %; serve p50/p99 latency"
WORKLOAD = ("pow2 sweep: 1D complex64 n=2^4..2^24, batch 2^26/n, contiguous, forward+backward; "
            "plus rank-2 4096x4096 and single n=2^24, forward+backward")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# kernel family -> (committed ncu traffic record, the sources its hash covers)
TRAFFIC_RECORDS = {
    "p2-tma": ("p2_tma_traffic.txt",
               ("stockham_pow2.cu", "gb_p2_stages.cuh", "gb_tma.cuh", "gb_kernels.h", "codelets.cuh")),
    "l2-fourstep": ("l2fs_traffic.txt",
                    ("l2fourstep.cu", "gb_p2_stages.cuh", "gb_tma.cuh", "gb_kernels.h", "codelets.cuh")),
}


def kernel_source_hash(family="p2-tma"):
    h = hashlib.sha256()
    for name in TRAFFIC_RECORDS[family][1]:
        with open(os.path.join(ROOT, "paper_2602_23525_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(family="p2-tma"):
    """DRAM bytes per launch of a kernel family from its committed ncu summary
    (``key: value`` lines), valid only if the kernel sources are unchanged since
    the capture."""
    if family not in TRAFFIC_RECORDS:
        return None
    path = os.path.join(ROOT, "profiles", TRAFFIC_RECORDS[family][0])
    if not os.path.exists(path):
        return None
    d = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    if d.get("kernel_hash") != kernel_source_hash(family):
        return None
    try:
        d["dram_bytes_per_launch"] = float(d["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None
    return d


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- workload

def workload_problems():
    """(label, dims, howmany, n_points_per_transform, count) of one step, per sign."""
    probs = []
    for n in fft_inputs.POW2_SWEEP:
        b = fft_inputs.SWEEP_POINTS // n
        probs.append((f"n=2^{int(math.log2(n))}", [(n, 1, 1)], [(b, n, n)], n, b))
    probs.append(("rank2 4096x4096", [(4096, 4096, 4096), (4096, 1, 1)], [], 4096 * 4096, 1))
    probs.append(("single n=2^24", [(2 ** 24, 1, 1)], [], 2 ** 24, 1))
    return probs


def flops_of(n_points, count):
    return 5.0 * n_points * math.log2(n_points) * count


def max_over_ranks(value, device):
    """The largest of every rank's value (a step time), through the process group
    when there is one."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_gflops(world, flops_per_rank_step, ms_per_step):
    """Whole-job throughput: every replica does the same step, timed by the slowest."""
    return world * flops_per_rank_step / (ms_per_step * 1e-3) / 1e9


# --------------------------------------------------------------------------- GPU arm

def run_gpu(args, rank, world):
    import torch

    from paper_2602_23525_gb300 import gbfft

    torch.cuda.set_device(args.local_rank)
    dev = torch.device("cuda", args.local_rank)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    flags = gbfft.FFT_ESTIMATE if args.estimate else gbfft.FFT_MEASURE

    x_np = fft_inputs.uniform_c64(fft_inputs.SWEEP_POINTS, fft_inputs.seed_for(1))
    xin = torch.from_numpy(x_np).to(dev)
    yout = torch.empty_like(xin)

    t0 = time.time()
    plans = []
    for label, dims, how, npts, count in workload_problems():
        for sign in (-1, 1):
            p = gbfft.Plan(dims, how, sign, flags)
            plans.append((label, sign, p, npts, count))
    plan_s = time.time() - t0

    def one_step(events=None):
        for i, (label, sign, p, npts, count) in enumerate(plans):
            if events is not None:
                events[i][0].record(stream)
            gbfft.fft_execute(p.handle, xin.data_ptr(), yout.data_ptr(), sptr)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plans]
          for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(args.local_rank)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed launches
    start.record(stream)
    for k in range(args.steps):
        one_step(ev[k])
    end.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(start.elapsed_time(end), dev)

    step_flops = sum(flops_of(npts, count) for _, _, _, npts, count in plans)
    step_bytes = sum(16.0 * npts * count for _, _, _, npts, count in plans)
    ms_per_step = total_ms / args.steps
    value = aggregate_gflops(world, step_flops, ms_per_step)

    # per-plan breakdown; the roofline is taken for the kernel family with the
    # largest share of the step (plans whose passes all use that family)
    per = []
    fam_alg, fam_pass, fam_ms, fam_launch = {}, {}, {}, {}
    for i, (label, sign, p, npts, count) in enumerate(plans):
        ms = statistics.median(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
        launches = p.launches
        alg = 16.0 * npts * count
        kinds = sorted({ln.strip().split(" ")[1] for ln in p.info.splitlines() if ln.strip().startswith("pass ")})
        fam = kinds[0] if len(kinds) == 1 else "+".join(kinds)
        per.append({"problem": label, "sign": sign, "ms": round(ms, 4),
                    "gflops": round(flops_of(npts, count) / (ms * 1e-3) / 1e9, 1),
                    "gbs_algorithmic": round(alg / (ms * 1e-3) / 1e9, 1), "launches": launches, "kernels": fam})
        fam_alg[fam] = fam_alg.get(fam, 0.0) + alg
        fam_pass[fam] = fam_pass.get(fam, 0.0) + alg * launches
        fam_ms[fam] = fam_ms.get(fam, 0.0) + ms
        fam_launch[fam] = fam_launch.get(fam, []) + [(launches, npts * count)]
    dom = max(fam_ms, key=lambda f: fam_ms[f])
    peak, peak_kind = peaks()
    # algorithmic bytes: 16 B per point per TRANSFORM (read once, written once);
    # the scratch round trips of multi-pass plans are not algorithmic
    achieved = fam_alg[dom] / (fam_ms[dom] * 1e-3) / 1e9
    pass_achieved = fam_pass[dom] / (fam_ms[dom] * 1e-3) / 1e9
    traffic = recorded_traffic(dom)
    traffic_exec = None
    if traffic:
        # DRAM bytes of one execution of the family's average plan: its launches
        # times the recorded bytes of one pass, scaled to the plan's points
        per_pt = traffic["dram_bytes_per_launch"] / float(traffic.get("points", 2 ** 26))
        runs = fam_launch[dom]
        traffic_exec = sum(nl * per_pt * pts for nl, pts in runs) / len(runs)
        alg_exec = sum(16.0 * pts for _, pts in runs) / len(runs)
    kernel_names = {"p2-tma": "gb_p2_kernel / gb_p2small_kernel (TMA power-of-two passes)",
                    "l2-fourstep": "gb_l2fs_kernel (the four-step in one persistent kernel, intermediate in L2)",
                    "cluster": "gb_cluster_kernel (one pass over a thread-block cluster)",
                    "stockham": "gb_stockham_kernel (generic pass)"}

    # end to end through the C ABI with host buffers (pinned), fewer steps
    e2e = None
    if not args.no_e2e:
        # host -> device copy of each problem's input, the transform, device ->
        # host copy of its result; consecutive problems rotate over a few
        # streams with their own device buffers, so copies overlap transforms
        nl = max(2, args.e2e_lanes)
        host_in = torch.from_numpy(x_np).pin_memory()
        host_out = [torch.empty_like(host_in).pin_memory() for _ in range(nl)]
        dbuf = [(xin, yout)] + [(torch.empty_like(xin), torch.empty_like(yout)) for _ in range(nl - 1)]
        lanes = [torch.cuda.Stream(dev) for _ in range(nl)]
        e2e_steps = max(1, min(args.steps, 2))

        def e2e_step():
            fork = torch.cuda.Event()
            fork.record(stream)
            for ls in lanes:
                ls.wait_event(fork)
            for i, (label, sign, p, npts, count) in enumerate(plans):
                m = npts * count
                ls, (di, do), ho = lanes[i % nl], dbuf[i % nl], host_out[i % nl]
                with torch.cuda.stream(ls):
                    di[:m].copy_(host_in[:m], non_blocking=True)
                    gbfft.fft_execute(p.handle, di.data_ptr(), do.data_ptr(), ls.cuda_stream)
                    ho[:m].copy_(do[:m], non_blocking=True)
            for ls in lanes:
                join = torch.cuda.Event()
                join.record(ls)
                stream.wait_event(join)

        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(a.elapsed_time(b) / e2e_steps, dev)
        nbytes = sum(8 * npts * count for _, _, _, npts, count in plans)
        # the host link's own ceiling: one host -> device and one device -> host
        # copy of the largest problem running at the same time on the two lanes
        mmax = max(npts * count for _, _, _, npts, count in plans)
        link_ms = []
        for rep in range(4):
            torch.cuda.synchronize()
            c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c.record(stream)
            for ls in lanes:
                ls.wait_event(c)
            with torch.cuda.stream(lanes[0]):
                dbuf[0][0][:mmax].copy_(host_in[:mmax], non_blocking=True)
            with torch.cuda.stream(lanes[1]):
                host_out[1][:mmax].copy_(dbuf[1][1][:mmax], non_blocking=True)
            for ls in lanes:
                join = torch.cuda.Event()
                join.record(ls)
                stream.wait_event(join)
            d.record(stream)
            torch.cuda.synchronize()
            if rep:
                link_ms.append(c.elapsed_time(d))
        link_gbs = 2 * 8 * mmax / (min(link_ms) * 1e-3) / 1e9
        e2e_gbs = 2 * nbytes / (e2e_ms * 1e-3) / 1e9
        e2e = {"value": round(aggregate_gflops(world, step_flops, e2e_ms), 2), "unit": "GFLOP/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": round(e2e_ms, 3),
               "pipeline": "%d streams in rotation, copies of one problem overlap the transforms of the "
                           "others" % nl,
               "host_link": {"achieved_gbs": round(e2e_gbs, 1), "peak_gbs": round(link_gbs, 1),
                             "frac": round(e2e_gbs / link_gbs, 3),
                             "peak_kind": "measured here: concurrent pinned H2D + D2H copies of %d bytes each "
                                          "on two streams" % (8 * mmax)}}

    launches = sum(p.launches for _, _, p, _, _ in plans) * args.steps
    result = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded uniform[-1,1) complex64)",
        "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (512 MiB per sweep point, 128 MiB "
                   "for rank-2 and 2^24 plus 128 MiB output)", "planner": "estimate" if args.estimate else
                   "measure", "parallelism": f"replicas x{world}",
                   "step_bytes_algorithmic": step_bytes, "step_flops": step_flops},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": (round(traffic_exec) if traffic_exec else None),
                     "traffic_over_algorithmic": (round(traffic_exec / alg_exec, 3) if traffic_exec else None),
                     "traffic_basis": ("DRAM bytes of one execution (all its launches) of the family's average "
                                       "plan: launches x the ncu bytes of one recorded pass (%s), scaled by points"
                                       % traffic["launch"]) if traffic else None,
                     "kernel": kernel_names.get(dom, dom),
                     "time_share": round(fam_ms[dom] / sum(fam_ms.values()), 4),
                     "unit_of_work": "16 B per point per transform (read once, written once; scratch round "
                                     "trips of multi-pass plans are not algorithmic)",
                     "peak_kind": f"{peak_kind} hbm_gbs (of measured)" if peak_kind == "measured"
                                  else f"{peak_kind} hbm_gbs",
                     "pass_achieved": round(pass_achieved, 1),
                     "pass_frac": round(pass_achieved / peak, 4),
                     "step_frac": round(step_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 4)},
        "clocks": clk, "gpu_launches": launches, "plan_seconds": round(plan_s, 2),
        "e2e": e2e, "per_problem": per,
    }
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    for _, _, p, _, _ in plans:
        p.destroy()
    return result


# --------------------------------------------------------------------------- oracle (CPU) arm

def cpu_sample(scale=1.0):
    """Bounded sample of the sweep for the FP64 oracle: (n, transforms)."""
    base = [(16, 4096), (256, 512), (4096, 8), (65536, 16), (2 ** 20, 1), (2 ** 24, 1)]
    return [(n, max(1, int(c * scale))) for n, c in base]


def time_oracle(sample, reps=1):
    import oracle
    threads = oracle.default_threads()
    flops, dt = 0.0, 0.0
    for n, c in sample:
        x = fft_inputs.uniform_c64(n * c, fft_inputs.seed_for(1))  # input generation is not timed
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.dft(x, [(n, 1, 1)], [(c, n, n)], -1, threads=threads)
            dt += time.perf_counter() - t0
            flops += flops_of(n, c)
    return flops, dt, threads


def cpu_baseline(target_s=12.0):
    # sixteen times the base sample (its largest transforms are threaded over
    # the batch only, sixteen of them keep the box's 16 host cores busy), run
    # three times: 10-30 s of oracle work
    sample = cpu_sample(16.0)
    flops, dt, threads = time_oracle(sample, reps=3)
    desc = ", ".join(f"{c} x n={n}" for n, c in sample)
    return {"value": round(flops / dt / 1e9, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"forward transforms {desc}, each batch three times (oracle: direct eq. (1) for "
                      f"n<=4096, recursive Cooley-Tukey above), {dt:.1f} s", "seconds": round(dt, 2)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    sample = [(16, 1024), (256, 128), (4096, 2), (65536, 4), (2 ** 20, 1)]
    for _ in range(args.warmup):
        time_oracle([(256, 64)])
    tot_f = tot_t = 0.0
    threads = 1
    for _ in range(args.steps):
        f, t, threads = time_oracle(sample)
        tot_f += f
        tot_t += t
    value = tot_f / tot_t / 1e9
    desc = ", ".join(f"{c} x n={n}" for n, c in sample)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * tot_t / args.steps, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded uniform[-1,1) complex64)",
            "config": {"workload": WORKLOAD, "sample_per_step": desc},
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": f"per step: forward transforms {desc}"},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_uneven(args):
    """The uneven-batch workload (sizes 1000, 2187, 3125, 7168, 10007, 65536 x 512,
    contiguous and transposed layouts) as one persistent group launch, and the
    same plans executed one after another, on one GPU."""
    import torch

    from paper_2602_23525_gb300 import gbfft
    batch = fft_inputs.UNEVEN_BATCH
    plans, ins, outs, flops = [], [], [], 0.0
    for i, n in enumerate(fft_inputs.UNEVEN_SIZES):
        dims, how = (fft_inputs.transposed_1d(n, batch) if n in fft_inputs.UNEVEN_TRANSPOSED
                     else fft_inputs.batched_1d(n, batch))
        plans.append(gbfft.Plan(dims, how, -1, gbfft.FFT_ESTIMATE if args.estimate else gbfft.FFT_MEASURE))
        x = torch.from_numpy(fft_inputs.gaussian_c64(n * batch, fft_inputs.seed_for(2, i))).cuda()
        ins.append(x)
        outs.append(torch.empty_like(x))
        flops += flops_of(n, batch)
    g = gbfft.fft_group_create([p.handle for p in plans])  # executor chosen by timing both
    mode = gbfft.fft_group_mode(g)
    s = torch.cuda.Stream()
    sp = s.cuda_stream
    ip, op = [t.data_ptr() for t in ins], [t.data_ptr() for t in outs]

    def timed(fn):
        with torch.cuda.stream(s):
            for _ in range(args.warmup):
                fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(args.steps):
                fn()
            b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    t_group = timed(lambda: gbfft.fft_group_execute(g, ip, op, sp))
    t_seq = timed(lambda: [gbfft.fft_execute(p.handle, i, o, sp) for p, i, o in zip(plans, ip, op)])
    status = gbfft.fft_group_status(g)
    # each executor on its own, for the record
    per_mode = {}
    for name, fl in (("persistent queue", gbfft.FFT_GROUP_PERSISTENT), ("graph of plan launches",
                                                                          gbfft.FFT_GROUP_GRAPH)):
        try:
            gm = gbfft.fft_group_create([p.handle for p in plans], fl)
        except gbfft.GbfftError as e:  # a plan step the persistent queue has no form for
            per_mode[name] = f"unsupported ({e.code})"
            continue
        per_mode[name] = round(timed(lambda: gbfft.fft_group_execute(gm, ip, op, sp)), 4)
        gbfft.fft_group_destroy(gm)
    nbytes = sum(16.0 * n * batch for n in fft_inputs.UNEVEN_SIZES)
    res = {"metric": METRIC, "workload": "uneven: sizes 1000, 2187, 3125, 7168, 10007, 65536 x 512, "
           "2187/7168/65536 transposed, forward, one group execution", "unit": "GFLOP/s",
           "executor_ms": per_mode,
           "group": {"ms": round(t_group, 4), "value": round(flops / (t_group * 1e-3) / 1e9, 1),
                     "gbs_algorithmic": round(nbytes / (t_group * 1e-3) / 1e9, 1),
                     "launches": gbfft.fft_group_launches(g),
                     "executor": "persistent queue" if mode == 1 else "graph of plan launches",
                     "status": status},
           "sequential": {"ms": round(t_seq, 4), "value": round(flops / (t_seq * 1e-3) / 1e9, 1),
                          "gbs_algorithmic": round(nbytes / (t_seq * 1e-3) / 1e9, 1),
                          "launches": sum(p.launches for p in plans)},
           "plans": [p.info for p in plans]}
    gbfft.fft_group_destroy(g)
    return res


def run_precision(args):
    """The tensor-core precision forms on the two precision workloads: batch 65536
    of n = 4096, and 256^3.  Each form (FP32 path, FP16, BF16, FP16 split, BF16
    split) is timed and its error against the FP64 oracle stated (sampled
    transforms for the batch, the whole cube for 256^3)."""
    import torch

    import oracle
    from paper_2602_23525_gb300 import gbfft
    forms = {"fp32": 0, "tc-fp16": gbfft.FFT_PREC_TC_FP16, "tc-bf16": gbfft.FFT_PREC_TC_BF16,
             "tc-fp16-split": gbfft.FFT_PREC_TC_FP16 | gbfft.FFT_PREC_SPLIT,
             "tc-bf16-split": gbfft.FFT_PREC_TC_BF16 | gbfft.FFT_PREC_SPLIT}
    cases = [("batch 65536 x n=4096", [(4096, 1, 1)], [(65536, 4096, 4096)], 4096, 65536),
             ("256^3", [(256, 65536, 65536), (256, 256, 256), (256, 1, 1)], [], 256 ** 3, 1)]
    out = {"metric": METRIC, "unit": "GFLOP/s", "workload": "precision forms", "cases": []}
    for label, dims, how, npts, count in cases:
        total = npts * count
        x_np = fft_inputs.uniform_c64(total, fft_inputs.seed_for(3, 0))
        x = torch.from_numpy(x_np).cuda()
        y = torch.empty_like(x)
        if count > 1:
            idx = [0, count // 3, count - 1]
            refs = {v: oracle.dft(x_np[v * npts:(v + 1) * npts], [(npts, 1, 1)], [], -1) for v in idx}
        else:
            refs = {0: oracle.dft(x_np, dims, [], -1, algo="ct")}
        res = {"case": label, "forms": {}}
        for name, fl in forms.items():
            p = gbfft.Plan(dims, how, -1, fl | gbfft.FFT_ESTIMATE)
            s = torch.cuda.current_stream().cuda_stream
            for _ in range(args.warmup):
                gbfft.fft_execute(p.handle, x.data_ptr(), y.data_ptr(), s)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(args.steps):
                gbfft.fft_execute(p.handle, x.data_ptr(), y.data_ptr(), s)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / args.steps
            yh = y.cpu().numpy()
            errs = []
            for v, ref in refs.items():
                yy = yh[v * npts:(v + 1) * npts].astype(np.complex128)
                errs.append(float(np.linalg.norm(yy - ref) / np.linalg.norm(ref)))
            res["forms"][name] = {"ms": round(ms, 4), "gflops": round(flops_of(npts, count) / (ms * 1e-3) / 1e9, 1),
                                  "gbs_algorithmic": round(16.0 * total / (ms * 1e-3) / 1e9, 1),
                                  "max_rel_l2_vs_fp64_oracle": max(errs),
                                  "passes": [ln.strip().split(" n=")[0] for ln in p.info.splitlines()
                                             if ln.strip().startswith("pass")]}
            p.destroy()
        out["cases"].append(res)
    return out


def run_planner(args):
    """Planner experiments on one GPU, every problem 2^24 complex points (128 MiB in
    and out, larger than L2), forward, timed with CUDA events:
      estimate_penalty -- each size planned in estimate mode (no timing) and in
        measure mode (candidates timed on the device), both executed: the paper's
        estimate-mode penalty (sec. 4.3) on this hardware;
      sizes_3600_3840_4096 -- the paper's observation (sec. 7) that lengths 3600
        and 3840 ran faster than 4096 on its CPU, at equal points per problem;
      prime_plans -- prime lengths with Rader (convolution length p - 1 or a
        padded power of two) against Bluestein (smallest 2^a3^b5^c7^d or power
        of two), each forced through a wisdom entry (sec. 4.2.5)."""
    import torch

    from paper_2602_23525_gb300 import gbfft
    total = 1 << 24
    x = torch.from_numpy(fft_inputs.uniform_c64(total, fft_inputs.seed_for(7))).cuda()
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    reps = max(5, args.steps)

    def timed(n, flags, wisdom=None):
        gbfft.fft_forget_wisdom()
        if wisdom:
            gbfft.fft_import_wisdom(wisdom)
        b = total // n
        t0 = time.time()
        p = gbfft.Plan([(n, 1, 1)], [(b, n, n)], -1, flags)
        plan_s = time.time() - t0
        for _ in range(3):
            gbfft.fft_execute(p.handle, x.data_ptr(), y.data_ptr(), s)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gbfft.fft_execute(p.handle, x.data_ptr(), y.data_ptr(), s)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        top = [ln.strip() for ln in p.info.splitlines()[1:] if ln.strip()]
        kind = top[0].split(" (")[0] if top else ""
        r = {"ms": round(ms, 4), "ns_per_point": round(ms * 1e6 / (n * b), 4),
             "gflops": round(flops_of(n, b) / (ms * 1e-3) / 1e9, 1),
             "gbs_algorithmic": round(16.0 * n * b / (ms * 1e-3) / 1e9, 1),
             "launches": p.launches, "plan_s": round(plan_s, 3), "plan": kind}
        p.destroy()
        return r

    sizes = [1 << e for e in range(4, 25)] + [1000, 2187, 3125, 3600, 3840, 7168, 10007, 12289]
    pen = []
    for n in sizes:
        est = timed(n, gbfft.FFT_ESTIMATE)
        mea = timed(n, gbfft.FFT_MEASURE)
        pen.append({"n": n, "batch": total // n, "estimate": est, "measure": mea,
                    "estimate_over_measure": round(est["ms"] / mea["ms"], 3)})
    e2 = {str(n): timed(n, gbfft.FFT_MEASURE) for n in (3600, 3840, 4096)}
    primes = []
    for pr in (1153, 7681, 12289, 65537, 10007, 40009):
        b = total // pr
        key = f"r1 n={pr} is=1 os=1 v=[({b},{pr},{pr})] ip=0\t"
        m2 = 1
        while m2 < 2 * pr - 1:
            m2 <<= 1
        r2 = 1
        while r2 < 2 * pr - 3:
            r2 <<= 1
        ms_ = 2 * pr - 1
        while not _smooth7(ms_):
            ms_ += 1
        opts = {}
        if _smooth13(pr - 1):
            opts[f"rader:{pr - 1}"] = None
        opts[f"rader:{r2}"] = None
        opts[f"blue:{ms_}"] = None
        opts[f"blue:{m2}"] = None
        row = {"p": pr, "batch": b}
        for o in opts:
            row[o] = timed(pr, gbfft.FFT_ESTIMATE, "gbfft-wisdom 1\n" + key + o + "\n")
        row["measured_choice"] = timed(pr, gbfft.FFT_MEASURE)
        primes.append(row)
    gbfft.fft_forget_wisdom()
    return {"metric": METRIC, "unit": "GFLOP/s", "workload": "planner experiments, 2^24 points per problem, "
            "forward", "reps": reps, "estimate_penalty": pen, "sizes_3600_3840_4096": e2, "prime_plans": primes}


def run_forms(args):
    """The transform forms beyond the complex sweep, on one GPU: real-input (r2c)
    and real-output (c2r) transforms of 2^26 real values (the half spectrum on the
    complex side), and in-place complex transforms of 2^26 points planned without
    scratch against the same problem out of place; CUDA events, forward unless
    stated."""
    import torch

    from paper_2602_23525_gb300 import gbfft
    total = 1 << 26
    s = torch.cuda.current_stream().cuda_stream
    reps = max(5, args.steps)

    def timed(plan, a, b):
        for _ in range(3):
            gbfft.fft_execute(plan, a.data_ptr(), b.data_ptr(), s)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gbfft.fft_execute(plan, a.data_ptr(), b.data_ptr(), s)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    xr = torch.from_numpy(np.random.default_rng(fft_inputs.seed_for(9)).uniform(-1, 1, total)
                          .astype(np.float32)).cuda()
    out = []
    for e in (12, 16, 20):
        n = 1 << e
        b = total // n
        h = n // 2 + 1
        yc = torch.empty(h * b, dtype=torch.complex64, device="cuda")
        zr = torch.empty(total, dtype=torch.float32, device="cuda")
        pf = gbfft.fft_plan_dft_r2c([(n, 1, 1)], [(b, n, h)], gbfft.FFT_MEASURE)
        pb = gbfft.fft_plan_dft_c2r([(n, 1, 1)], [(b, h, n)], gbfft.FFT_MEASURE)
        for kind, plan, a, c in (("r2c", pf, xr, yc), ("c2r", pb, yc, zr)):
            ms = timed(plan, a, c)
            out.append({"form": kind, "n": n, "batch": b, "ms": round(ms, 4),
                        "gflops": round(2.5 * n * math.log2(n) * b / (ms * 1e-3) / 1e9, 1),
                        "gbs_algorithmic": round(gbfft.fft_plan_bytes(plan) / (ms * 1e-3) / 1e9, 1),
                        "launches": gbfft.fft_plan_launches(plan)})
            gbfft.fft_destroy(plan)
        del yc, zr
    del xr
    x = torch.from_numpy(fft_inputs.uniform_c64(total, fft_inputs.seed_for(10))).cuda()
    y = torch.empty_like(x)
    for e in (16, 20, 24):
        n = 1 << e
        b = total // n
        how = [(b, n, n)] if b > 1 else []
        pi = gbfft.Plan([(n, 1, 1)], how, -1, gbfft.FFT_INPLACE | gbfft.FFT_ESTIMATE)
        po = gbfft.Plan([(n, 1, 1)], how, -1, gbfft.FFT_ESTIMATE)
        ms_i = timed(pi.handle, x, x)
        ms_o = timed(po.handle, x, y)
        out.append({"form": "in place, no scratch", "n": n, "batch": b, "ms": round(ms_i, 4),
                    "gflops": round(flops_of(n, b) / (ms_i * 1e-3) / 1e9, 1),
                    "scratch_bytes": gbfft.fft_plan_scratch_bytes(pi.handle), "launches": pi.launches,
                    "out_of_place_ms": round(ms_o, 4),
                    "out_of_place_scratch_bytes": gbfft.fft_plan_scratch_bytes(po.handle)})
        pi.destroy()
        po.destroy()
    return {"metric": METRIC, "unit": "GFLOP/s", "workload": "transform forms: real data and in place, "
            "2^26 values per problem", "reps": reps, "forms": out}


def _smooth7(m):
    for q in (2, 3, 5, 7):
        while m % q == 0:
            m //= q
    return m == 1


def _smooth13(m):
    for q in (2, 3, 5, 7, 11, 13):
        while m % q == 0:
            m //= q
    return m == 1


def run_serving(args):
    """The serving workload: requests of mixed shapes (rank 1-3), batches and signs
    with Poisson arrivals, admitted by a 40 GB work-buffer budget.  The arrival
    rate is 70% of the closed-loop capacity measured on the first requests.
    Host buffers are pinned; requests share one input and one output pool."""
    import torch

    from paper_2602_23525_gb300 import gbfft
    reqs = fft_inputs.serving_requests(args.requests, fft_inputs.seed_for(5))
    max_elems = max(int(np.prod(sh)) * b for sh, b, _ in reqs)
    pool_in = torch.from_numpy(fft_inputs.uniform_c64(max_elems, fft_inputs.seed_for(5, 1))).pin_memory()
    pool_out = torch.empty_like(pool_in).pin_memory()
    pin, pout = pool_in.data_ptr(), pool_out.data_ptr()

    def run(subset, rate):
        server = gbfft.fft_server_create(fft_inputs.SERVING_BUDGET, args.streams)
        t_start = gbfft.fft_server_now(server)
        arrivals = (fft_inputs.poisson_arrivals(len(subset), rate, fft_inputs.seed_for(5, 2))
                    if rate else np.zeros(len(subset)))
        for (shape, batch, sign), at in zip(subset, arrivals):
            when = t_start + float(at)
            while rate and gbfft.fft_server_now(server) < when:
                d = when - gbfft.fft_server_now(server)
                if d > 2e-4:
                    time.sleep(d - 1e-4)
            gbfft.fft_server_submit(server, shape, batch, sign, pin, pout, when)
        gbfft.fft_server_drain(server, 3600.0)
        st = gbfft.fft_server_stats(server)
        gbfft.fft_server_destroy(server)
        return st

    calib = reqs[: max(1, min(len(reqs), args.requests // 10))]
    run(calib[: min(50, len(calib))], 0)  # warm the caches the loop does not own (first plans, context)
    closed = run(calib, 0)
    rate = args.rate if args.rate else 0.7 * closed["requests_per_s"]
    open_ = run(reqs, rate)
    return {"metric": METRIC, "workload": "serving: %d requests, Poisson arrivals at %.1f/s (0.7 x closed-loop "
            "capacity %.1f/s), n 2^6..2^20 (80%%) or non-power-of-two 100..1e5, rank 1/2/3, batch 1..256, "
            "sign +-1, 40 GB budget, %d streams" % (len(reqs), rate, closed["requests_per_s"], args.streams),
            "unit": "s", "p50_latency_s": open_["p50_latency_s"], "p99_latency_s": open_["p99_latency_s"],
            "throughput_gflops": open_["gflops"], "throughput_requests_per_s": open_["requests_per_s"],
            "higher_is_better": False, "open_loop": open_, "closed_loop": closed,
            "host_buffers": "pinned, shared pools (inputs read from one pool, outputs written to one pool)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="sweep", choices=["sweep", "uneven", "serving", "precision", "planner", "forms"],
                    help="sweep: the benchmark step; uneven / serving: extra workloads (their own line)")
    ap.add_argument("--requests", type=int, default=100000, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=0.0, help="serving: arrivals per second (0: 0.7 x capacity)")
    ap.add_argument("--streams", type=int, default=4, help="serving: streams")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbfft", choices=["gbfft", "reference"])
    ap.add_argument("--estimate", action="store_true", help="plan with FFT_ESTIMATE instead of measuring")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-lanes", type=int, default=2, help="e2e: streams the problems rotate over")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="unused; kept for the command line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    args.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload in ("uneven", "serving", "precision", "planner", "forms"):
        if rank == 0:
            fn = {"uneven": run_uneven, "serving": run_serving, "precision": run_precision,
                  "planner": run_planner, "forms": run_forms}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(args.local_rank)
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
