"""Benchmark of GB300 lambda-thinning: one JSON line on stdout (rank 0).

Workload (a step): one batch of 64 synthetic 512x512 u8 images, each thinned
at lambda in {0, 5, 20} (192 jobs), in one thin_batch call -- one persistent
device-driven launch.  Images are restored from pristine device copies and L2
is flushed (a 512 MiB write) before every timed step, outside the timed
region.  Timing: CUDA events on the launching stream around each step,
barrier + synchronize around the K timed steps, max over ranks.  The line
also carries the metric's other two parts, measured in the same run at N = 1:
`large` (4096x4096 u8 and 8192x8192 u16 at lambda 0 and 30 through thin_run:
ms, Gpix-sweeps/s and HBM-roofline fractions) and `serve` (Poisson arrivals
through the serving API: the capacity (the whole mix queued at once), a
saturated run, and Poisson arrivals at half the capacity: images/s, p50/p99
latency, and the single-image service time of the mix).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload large|uneven|serve   (the other configurations)

--workload large: the large images with the tiled engine beside the wide
resident mode and a halo sweep.  --workload uneven: 1024 u8 images with
sides log-uniform in [64, 2048] and lambda in {0, 10, 25}, one thin_batch
call against one thin_run call per image.  --workload serve: Poisson
arrivals of u8/u16 images with sides log-uniform in [128, 4096] through the
serving API under a 40 GB budget, at 1k..50k requests/s and at 25, 50 and
90 % of the measured capacity, against a plain one-image-at-a-time path;
p50/p99 latency and images/s per arrival rate.  Lambda applies to pixel
values as given, for u8 and u16 alike.

--impl reference times the CPU oracle (the plain sequential subfield
schedule) on this host's cores over a bounded sample of the same jobs.
Multi-GPU: one process per GPU under torchrun; every rank thins its own batch
(images are independent, no collective on the data path) -> weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "λ-thinned images/s (512² u8) & Gpix-sweeps/s vs HBM roofline; p99 latency"
N_IMAGES = 64
LAMBDAS = (0, 5, 20)
SIDE = 512
PAPER_IMG_PER_S = 125.0  # Sec. 5.2 / abstract: lambda-skeleton, 512^2 MRI, 2x Xeon E5405 (context only)
CSRC = os.path.join(ROOT, "paper_1603_09180_gb300", "csrc")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")


# The sources of the dominant kernel (k_resident): its recorded DRAM traffic is used only while
# these are unchanged since the ncu capture.
KERNEL_SOURCES = ("thin_resident.cu", "thin_simd.cuh", "thin_common.cuh", "thin_internal.h")


def kernel_source_hash() -> str:
    """Hash of the dominant kernel's sources with comments and blank space removed
    (edits to comments keep the recorded counters valid)."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(CSRC, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).encode())
    return h.hexdigest()[:16]


ISSUE_FILE = os.path.join(ROOT, "profiles", "roofline_issue.json")


def issue_roofline(tested, ms_per_step, peaks):
    """The resident engine's instruction-issue roofline.  Peak: 152 SMs x 4 schedulers x 1 warp-instruction
    per clock x the SM clock (MEASURED_PEAKS.json sm_max_mhz).  Achieved: warp-instructions per point test,
    from an ncu count of smsp__inst_executed.sum over the point tests of the same launch (recorded in
    profiles/roofline_issue.json for the kernel sources of that hash), times this launch's point tests,
    over its device time.  None when the record does not match the current sources."""
    mhz = float(peaks.get("sm_max_mhz") or 2070.0)
    peak = 152 * 4 * mhz * 1e6
    try:
        rec = json.load(open(ISSUE_FILE))
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return {"bound": "alu", "achieved": None, "peak": round(peak / 1e12, 4), "unit": "T warp-instructions/s",
                "frac": None, "note": "instruction count not recorded for the current kernel sources"}
    ipt = float(rec["warp_instructions_per_point_test"])
    achieved = ipt * tested / (ms_per_step / 1e3)
    return {"bound": "alu", "achieved": round(achieved / 1e12, 4), "peak": round(peak / 1e12, 4),
            "unit": "T warp-instructions/s", "frac": round(achieved / peak, 4),
            "warp_instructions_per_point_test": ipt, "source": "profiles/roofline_issue.json",
            "peak_derivation": "152 SMs x 4 warp schedulers x 1 warp-instruction/clock x %.0f MHz" % mhz}


def workload_images():
    from paper_1603_09180_gb300.synth import value_noise_image
    return [value_noise_image(SIDE, SIDE, "u8", seed=s) for s in range(N_IMAGES)]


def jobs_of(images):
    return [(k, lam) for k in range(len(images)) for lam in LAMBDAS]


# ------------------------------------------------------------------ oracle leg

def _oracle_job(args):
    img, lam = args
    import oracle
    t = time.perf_counter()
    oracle.thin(img, lam)
    return time.perf_counter() - t


def oracle_sample(images, n_jobs: int, workers: int):
    """Times the CPU oracle on the first n_jobs jobs (cycling lambda) with a
    spawn pool of `workers` processes.  Returns (jobs/s, wall seconds)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    todo = [(images[(k // len(LAMBDAS)) % len(images)], LAMBDAS[k % len(LAMBDAS)]) for k in range(n_jobs)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_job, todo, chunksize=1)
    wall = time.perf_counter() - t0
    return n_jobs / wall, wall


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.environ.get("THIN_BENCH_CLOCKS_CSV")  # optional: keep the raw samples in this file

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
            if self.path:
                with open(self.path, "w") as f:
                    f.write(self.FIELDS + "\n" + "\n".join(self.lines) + "\n")

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ GPU leg

def rounds_profile(sts, bins: int = 8) -> dict:
    """Rounds each job ran up to and including its last change (the quiet phases of the stop rule
    not counted): their spread, and a histogram in `bins` equal-width bins from 0 to the maximum.
    A long upper tail is time in which few images keep the engine busy."""
    r = sorted(s["last_change_phase"] // 4 + 1 for s in sts)
    if not r:
        return {"jobs": 0}
    top = r[-1]
    width = max(1, -(-top // bins))
    counts = [0] * bins
    for v in r:
        counts[min(bins - 1, v // width)] += 1
    q = lambda f: r[min(len(r) - 1, int(f * len(r)))]
    return {"jobs": len(r), "min": r[0], "p50": q(0.5), "p90": q(0.9), "max": top,
            "mean": round(sum(r) / len(r), 1), "bin_width": width, "hist": counts}


def max_over_ranks(vals, world: int, device=None):
    """Element-wise max of a list of floats over all ranks (identity at world 1)."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def run_gpu(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1603_09180_gb300 import thin

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    thin.load()
    images = workload_images()
    jobs = jobs_of(images)
    n_jobs = len(jobs)

    # inputs of the large-image and serving figures (rank 0, N = 1), made in a spawn pool before any device work
    extra = rank == 0 and world == 1
    large_imgs = _gen_pool(large_specs(), 2) if extra and not args.no_large else None
    serve_pool = serve_lams = None
    if extra and not args.no_serve:
        specs, serve_lams = serve_pool_specs(args.serve_pool)
        serve_pool = _gen_pool(specs, host_cores())

    # CPU baseline (rank 0, N = 1 only) before any device work, in a spawn pool
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        n = max(len(LAMBDAS), (cores // len(LAMBDAS)) * len(LAMBDAS))
        v, wall = oracle_sample(images, n, min(cores, n))
        cpu = {"value": v, "unit": "images/s", "cores": min(cores, n), "kind": "oracle",
               "sample": "%d of the %d jobs (images 0..%d x lambda %s), one process per job, %.1f s wall" % (
                   n, n_jobs, (n - 1) // len(LAMBDAS), list(LAMBDAS), wall)}

    pristine = torch.from_numpy(np.stack([images[k] for k, _ in jobs])).to(dev)  # (192, 512, 512)
    work = torch.empty_like(pristine)
    lams = [lam for _, lam in jobs]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    opts = dict(tile=args.tile or None, halo=args.halo, kernel=args.kernel)

    plan = thin.BatchPlan([work[k] for k in range(n_jobs)], lams, **opts)

    def one_step():
        plan.run(stream)

    # stats pass: algorithmic units of one step (deterministic)
    work.copy_(pristine)
    sts, rc = plan.run(stream, stats=True)
    assert rc == 0, rc
    # a point is tested at most once per round (in the phase of its parity) and only while one of
    # its neighbours moves: tested points = active pixel-rounds
    pix_rounds = float(sum(s["tested"] for s in sts))
    full_rounds = float(sum(SIDE * SIDE * s["phases"] / 4.0 for s in sts))
    alg_bytes = pix_rounds * 2.0  # 1 read + 1 write of a u8 pixel per active pixel-round
    launches_per_step = 2 if args.kernel == "tiled" else 1

    for _ in range(args.warmup):
        work.copy_(pristine)
        one_step()
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            work.copy_(pristine)
            flush.fill_(k & 0xff)  # evict L2 (larger than the 126 MB L2)
            starts[k].record(stream)
            one_step()
            ends[k].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)

    # end to end through the C-ABI with host buffers.  Every step copies its 192 inputs in from pinned host
    # memory, thins them with one thin_batch call and copies the 192 results back.  Two device buffers and
    # one copy stream per direction let step k's kernel run while step k+1's inputs arrive and step k-1's
    # results leave; L2 is flushed before every step's kernel, inside the timed region.
    host_in = torch.from_numpy(np.stack([images[k] for k, _ in jobs])).pin_memory()
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    bufs = [work, torch.empty_like(work)]
    plans = [plan, thin.BatchPlan([bufs[1][k] for k in range(n_jobs)], lams, **opts)]
    h2d_s, d2h_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_pipelined(n):
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        t0.record(h2d_s)
        for k in range(n):
            b = k % 2
            if k >= 2:
                h2d_s.wait_event(ev_out[b])  # the buffer's previous results have left
            with torch.cuda.stream(h2d_s):
                bufs[b].copy_(host_in, non_blocking=True)
            ev_in[b].record(h2d_s)
            stream.wait_event(ev_in[b])
            flush.fill_(k & 0xff)
            plans[b].run(stream)
            ev_done[b].record(stream)
            d2h_s.wait_event(ev_done[b])
            with torch.cuda.stream(d2h_s):
                host_out[b].copy_(bufs[b], non_blocking=True)
            ev_out[b].record(d2h_s)
        t1.record(d2h_s)
        torch.cuda.synchronize(dev)
        return t0.elapsed_time(t1) / n

    n_e2e = max(4, args.steps)
    e2e_pipelined(2)  # warm-up
    e2e_step_ms_local = e2e_pipelined(n_e2e)
    copy_ok = bool(torch.equal(host_out[(n_e2e - 1) % 2], bufs[(n_e2e - 1) % 2].cpu()))

    # the same, one step at a time (no overlap between steps), for comparison
    e2e_serial_ms = []
    for k in range(max(3, args.steps // 2) + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(k & 0xff)
        e0.record(stream)
        work.copy_(host_in, non_blocking=True)
        one_step()
        host_out[0].copy_(work, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if k:  # first one is a warm-up
            e2e_serial_ms.append(e0.elapsed_time(e1))

    # the paper's own operator, the lambda-skeleton (Sec. 2.2), on the same 192 jobs: the figure that
    # compares one to one with the paper's 125 images/s (outside the timed steps; `value` stays lambda-thinning)
    plan_sk = thin.BatchPlan([work[k] for k in range(n_jobs)], lams, op="skeleton", **opts)
    with ClockSampler(local_rank) as clk_k:
        ms_sk = statistics.median(_timed(lambda: plan_sk.run(stream), lambda: work.copy_(pristine), flush, stream, 5, 3))
    skeleton = {"images_per_s": round(n_jobs / (ms_sk / 1e3), 1), "ms_per_step": round(ms_sk, 4), "steps": 5,
                "warmup": 3, "x_paper": round(n_jobs / (ms_sk / 1e3) / PAPER_IMG_PER_S, 1), "clocks": clk_k.summary(),
                "note": "the same 192 jobs under the lambda-skeleton (lambda-deletable and not lambda-end), one "
                        "thin_batch call per step, L2 flushed before each; median of 5"}

    # the other two parts of the metric: large single images (Gpix-sweeps/s against the HBM roofline) and
    # serving (images/s and p50/p99 latency below and at capacity)
    large = serve = None
    if large_imgs is not None:
        with ClockSampler(local_rank) as clk_l:
            res_l, peak_l, _ = large_measure(large_imgs, 3, 3, flush, stream)
        large = {"cases": res_l, "clocks": clk_l.summary(), "steps": 3, "warmup": 3,
                 "note": "thin_run on the default engine; L2 flushed before every timed run; frac over active "
                         "pixel-rounds, frac_full over every pixel of every round"}
    if serve_pool is not None:
        with ClockSampler(local_rank) as clk_s:
            serve = serve_summary(serve_pool, serve_lams, dev, args.serve_slots, args.serve_queue, 3.0)
        serve["clocks"] = clk_s.summary()
        serve["config"] = ("Poisson arrivals, sides log-uniform [128, 4096], u8/u16 1:1, lambda {0, 10} on pixel "
                           "values as given, %d-image pool cycled, %d GB budget, %d slots"
                           % (args.serve_pool, SERVE_BUDGET >> 30, args.serve_slots))

    total_ms, e2e_step_ms, e2e_serial_step_ms = max_over_ranks(
        [total_ms, e2e_step_ms_local, sum(e2e_serial_ms) / len(e2e_serial_ms)], world, dev)
    if rank != 0:
        return None

    ms_per_step = total_ms / args.steps
    value = world * n_jobs / (total_ms / args.steps / 1e3)
    achieved = alg_bytes / (ms_per_step / 1e3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured"
    if not peak:
        peak, peak_src = 6800.0, "fallback"
    traffic = None
    try:
        tr = json.load(open(TRAFFIC_FILE))
        if tr.get("source_hash") == kernel_source_hash() and tr.get("workload") == "batch192":
            traffic = tr.get("traffic_bytes_per_launch")
    except Exception:
        pass
    clocks = clk.summary()
    issue = issue_roofline(pix_rounds, ms_per_step, peaks)
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "images/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic (seeded value-noise + dark lines; the paper's MRI image is not available)",
        "config": {"workload": "batch of %d images 512x512 u8 x lambda {0,5,20} = %d jobs, one thin_batch call"
                               % (N_IMAGES, n_jobs), "jobs_per_gpu": n_jobs,
                   "l2": "flushed before every timed step (512 MiB write)", "parallelism": "replicas x%d" % world},
        "gpix_sweeps_per_s": round(world * pix_rounds / (ms_per_step / 1e3) / 1e9, 3),
        "gpix_sweeps_full_per_s": round(world * full_rounds / (ms_per_step / 1e3) / 1e9, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 5), "traffic": traffic,
                     "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "note": "achieved = 2 B x active pixel-rounds (point tests) / thin_batch device time; "
                             "the engine keeps each image in shared memory, so its real limit is instruction "
                             "issue, not HBM (profiles/)"},
        "roofline_issue": issue,
        "e2e": {"value": round(world * n_jobs / (e2e_step_ms / 1e3), 2), "unit": "images/s",
                "h2d_bytes_per_step": int(host_in.numel()), "d2h_bytes_per_step": int(host_out[0].numel()),
                "ms_per_step": round(e2e_step_ms, 4), "steps": n_e2e,
                "how": "thin_batch on 192 images per step with the step's H2D and D2H inside the timed region; "
                       "two device buffers overlap step k's kernel with step k+1's H2D and step k-1's D2H",
                "serial_value": round(world * n_jobs / (e2e_serial_step_ms / 1e3), 2),
                "serial_note": "one step at a time: H2D, thin, D2H, no overlap between steps",
                "copy_check": copy_ok,
                "copy_check_note": "the D2H result equals the device result (a check of the copy, not of parity)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "paper_context": {"images_per_s": PAPER_IMG_PER_S, "note": "lambda-skeleton on a 512^2 MRI, 8 Xeon cores"},
        "step_ms": {"min": round(min(step_ms), 4), "p50": round(statistics.median(step_ms), 4),
                    "p99": round(sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))], 4),
                    "max": round(max(step_ms), 4)},
        "rounds": rounds_profile(sts),
        "engine": args.kernel,
        "skeleton": skeleton,
        "large": large,
        "serve": serve,
    }
    return line


def run_reference(args, rank: int, world: int):
    """The reference arm: the CPU oracle as it stands on this host's cores."""
    if rank != 0:
        return None
    images = workload_images()
    cores = host_cores()
    per_step = max(len(LAMBDAS), (cores // len(LAMBDAS)) * len(LAMBDAS))
    for _ in range(min(args.warmup, 1)):
        oracle_sample(images, len(LAMBDAS), len(LAMBDAS))
    walls = []
    for _ in range(args.steps):
        _, wall = oracle_sample(images, per_step, min(cores, per_step))
        walls.append(wall)
    total = sum(walls)
    value = per_step * args.steps / total
    return {
        "metric": METRIC, "value": round(value, 3), "unit": "images/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "impl": "reference",
        "data": "synthetic (seeded value-noise + dark lines)",
        "config": {"workload": "batch of 64 images 512x512 u8 x lambda {0,5,20} = 192 jobs; each step a sample "
                               "of %d jobs on the host cores" % per_step},
        "cpu_baseline": {"kind": "oracle", "cores": min(cores, per_step), "value": round(value, 3),
                         "unit": "images/s", "sample": "%d jobs per step, one process per job" % per_step},
        "e2e": {"value": round(value, 3), "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------------ other configurations

def _gen_pool(specs, workers):
    """Generates images for (h, w, dtype, seed[, vmax]) specs in a spawn pool (before any device work)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, workers)) as pool:
        return pool.map(_gen_one, specs, chunksize=1)


def _gen_one(spec):
    from paper_1603_09180_gb300.synth import value_noise_image
    h, w, dt, seed = spec[:4]
    vmax = spec[4] if len(spec) > 4 else None
    return value_noise_image(h, w, dt, seed=seed, vmax=vmax)


def _to_dev(a, dev):
    import numpy as np
    import torch
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).to(dev).view(torch.uint16)
    return torch.from_numpy(a).to(dev)


def _peak_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _timed(fn, restore, flush, stream, steps, warmup):
    """CUDA-event times (ms) of `steps` calls of fn, each after restore() and an L2 flush."""
    import torch
    for _ in range(warmup):
        restore()
        fn()
    torch.cuda.synchronize()
    ms = []
    for k in range(steps):
        restore()
        flush.fill_(k & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


LARGE_CASES = [(4096, 4096, "u8", 255, (0, 30)), (8192, 8192, "u16", 4095, (0, 30))]


def large_specs():
    return [(h, w, dt, 1603 + i, vmax) for i, (h, w, dt, vmax, _) in enumerate(LARGE_CASES)]


def large_measure(imgs, steps, warmup, flush, stream, compare_tiled=False, halo_sweep=False):
    """4096^2 u8 and 8192^2 u16 at lambda 0 and 30 on the default engine (thin_run): ms, sweep rates over
    active and over all pixels, and the HBM roofline (2 sizeof(T) bytes per active pixel-round)."""
    import torch
    from paper_1603_09180_gb300 import thin
    dev = flush.device
    peak, src = _peak_hbm()
    results = []
    for (h, w, dt, vmax, lams), img in zip(LARGE_CASES, imgs):
        pristine = _to_dev(img, dev)
        work = pristine.clone()
        es = work.element_size()
        for lam in lams:
            work.copy_(pristine)
            st = thin.run(work, lam)  # the default engine: wide resident if the image fits, else tiled
            engine = "tiled" if st["tiles_visited"] else "resident (wide)"
            tw, th, H = 64, 32, 8
            ms = _timed(lambda: thin.run(work, lam, stats=False), lambda: work.copy_(pristine),
                        flush, stream, steps, warmup)
            t = statistics.median(ms) / 1e3
            # pixel-rounds over active tiles (tiled) or tested pixel-rounds (resident: a point is tested
            # at most once per round, and only while a neighbour moved)
            active = st["tiles_visited"] * tw * th * H / 4.0 if st["tiles_visited"] else float(st["tested"])
            full = w * h * st["phases"] / 4.0
            r = {"image": "%dx%d %s" % (w, h, dt), "lambda": lam, "engine": engine, "ms": round(t * 1e3, 3),
                 "phases": st["phases"], "tiles_visited": st["tiles_visited"], "tested": st["tested"],
                 "gpix_sweeps_per_s": round(active / t / 1e9, 2),
                 "gpix_sweeps_full_per_s": round(full / t / 1e9, 2),
                 "point_tests_per_s_g": round(st["tested"] / t / 1e9, 2),
                 "achieved_gbs": round(2 * es * active / t / 1e9, 1),
                 "frac": round(2 * es * active / t / 1e9 / peak, 4),
                 "frac_full": round(2 * es * full / t / 1e9 / peak, 4)}
            if compare_tiled and engine != "tiled":  # the tiled engine on the same image, for comparison
                ms_t = _timed(lambda: thin.run(work, lam, kernel="tiled", stats=False),
                              lambda: work.copy_(pristine), flush, stream, max(1, steps // 2), 1)
                r["tiled_ms"] = round(statistics.median(ms_t), 3)
            results.append(r)
        if halo_sweep and dt == "u8":  # the tiled engine's halo depth, 4096^2 u8, lambda 30
            sweep = {}
            for H in (3, 4, 6, 8, 12, 16):
                ms = _timed(lambda: thin.run(work, 30, kernel="tiled", tile=(64, 32) if H <= 8 else (64, 48),
                                             halo=H, stats=False),
                            lambda: work.copy_(pristine), flush, stream, 1, 1)
                sweep[H] = round(ms[0], 3)
            results[-1]["tiled_halo_sweep_ms"] = sweep
        del pristine, work
        torch.cuda.empty_cache()
    return results, peak, src


def run_large(args):
    """Large single images on the default engine (the wide resident mode or the tiled engine)."""
    import torch
    from paper_1603_09180_gb300 import thin
    imgs = _gen_pool(large_specs(), 2)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    thin.load()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    with ClockSampler(0) as clk:
        results, peak, src = large_measure(imgs, args.steps, args.warmup, flush, stream, compare_tiled=True,
                                           halo_sweep=True)
    head = results[1]
    return {"metric": "Gpix-sweeps/s (4096^2 u8, lambda 30)", "value": head["gpix_sweeps_per_s"],
            "unit": "Gpix-sweeps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "u8/u16", "data": "synthetic", "workload": "large",
            "config": {"workload": "4096x4096 u8 and 8192x8192 u16 (0..4095), lambda 0 and 30, default engine "
                                   "(wide resident where the image fits the GPU's shared memory, else tiled 64x32, "
                                   "halo 8)", "l2": "flushed before every timed run"},
            "roofline": {"bound": "hbm", "achieved": head["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": head["frac"], "peak_source": src,
                         "note": "2 B (u8) or 4 B (u16) per pixel-round over active tiles (tiled) or per tested "
                                 "pixel-round (resident)"},
            "cases": results, "clocks": clk.summary()}


def run_uneven(args):
    """1024 uneven u8 images: one thin_batch call against one thin_run per image."""
    import numpy as np
    import torch
    from paper_1603_09180_gb300 import synth, thin
    specs = synth.uneven_batch_specs(args.uneven_n)
    imgs = _gen_pool([(h, w, "u8", seed) for h, w, lam, seed in specs], host_cores())
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    thin.load()
    lams = [lam for _, _, lam, _ in specs]
    pristine = [_to_dev(a, dev) for a in imgs]
    work = [p.clone() for p in pristine]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def restore():
        for a, b in zip(work, pristine):
            a.copy_(b)

    plan = thin.BatchPlan(work, lams)
    restore()
    sts, rc = plan.run(stream, stats=True)
    assert rc == 0, rc
    batch_out = [t.clone() for t in work]
    gplan = thin.GraphPlan(work, lams)
    with ClockSampler(0) as clk:
        ms_batch = _timed(lambda: plan.run(stream), restore, flush, stream, args.steps, args.warmup)
        ms_graph = _timed(lambda: gplan.run(stream), restore, flush, stream, args.steps, args.warmup)
        same_graph = all(torch.equal(a, b) for a, b in zip(work, batch_out))

        def per_image():
            for t, lam in zip(work, lams):
                thin.run(t, lam, stats=False)
        restore()
        per_image()
        same = all(torch.equal(a, b) for a, b in zip(work, batch_out))
        ms_single = _timed(per_image, restore, flush, stream, max(1, args.steps // 2), 1)
    n = len(specs)
    px = sum(h * w for h, w, _, _ in specs)
    tb, ts = statistics.median(ms_batch) / 1e3, statistics.median(ms_single) / 1e3
    return {"metric": "images/s, uneven batch of %d u8 images (sides 64..2048)" % n, "value": round(n / tb, 1),
            "unit": "images/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "u8", "data": "synthetic", "workload": "uneven",
            "config": {"workload": "%d u8 images, w and h log-uniform in [64, 2048], lambda in {0, 10, 25}" % n,
                       "megapixels": round(px / 1e6, 1), "l2": "flushed before every timed run"},
            "batch_ms": round(tb * 1e3, 2), "graph_plan_ms": round(statistics.median(ms_graph), 2),
            "graph_results_equal": same_graph, "per_image_launch_ms": round(ts * 1e3, 2),
            "per_image_images_per_s": round(n / ts, 1), "speedup_vs_per_image": round(ts / tb, 2),
            "results_equal": same, "max_phases": max(s["phases"] for s in sts),
            "mpix_per_s": round(px / tb / 1e6, 1), "clocks": clk.summary()}


SERVE_BUDGET = 40 << 30


def serve_pool_specs(pool_n):
    from paper_1603_09180_gb300 import synth
    _, spec0 = synth.serve_trace(1000.0, pool_n)
    return [(h, w, dt, seed) for h, w, dt, lam, seed in spec0], [lam for h, w, dt, lam, seed in spec0]


def _drive(rate, seconds, pool, submit, drain):
    """Poisson arrivals at `rate` for `seconds` (images cycled from the pool, lambda from the trace,
    applied to pixel values as given); returns latency and throughput figures."""
    from paper_1603_09180_gb300 import synth
    t_arr, spec = synth.serve_trace(rate, int(rate * seconds) + 1, seed=int(rate))
    sub_t, lat, rejected = {}, [], 0
    t0 = time.perf_counter()
    for k, ta in enumerate(t_arr):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        ts = time.perf_counter()
        tk = submit(pool[k % len(pool)], spec[k][3])
        if tk is None:
            rejected += 1
        else:
            sub_t[tk] = ts
    t_sub_end = time.perf_counter()
    done_t = drain(len(sub_t))
    for tk, td in done_t.items():
        lat.append(td - sub_t[tk])
    t_end = max(done_t.values()) if done_t else t_sub_end
    # steady state: completions while requests keep arriving, after the first quarter of the window
    w0 = t0 + 0.25 * (t_sub_end - t0)
    in_window = sum(1 for td in done_t.values() if w0 <= td <= t_sub_end)
    lat.sort()
    pct = lambda q: round(1e3 * lat[min(len(lat) - 1, int(q * len(lat)))], 2) if lat else None
    return {"rate_per_s": round(rate, 1), "offered": len(t_arr), "completed": len(lat), "rejected": rejected,
            "images_per_s": round(len(lat) / (t_end - t0), 1),
            "steady_images_per_s": round(in_window / max(1e-9, t_sub_end - w0), 1),
            "p50_ms": pct(0.5), "p99_ms": pct(0.99), "seconds": round(t_sub_end - t0, 2)}


def serve_served(pool, rate, seconds, slots, queue):
    """Poisson arrivals through thin_serve_* (continuous batching)."""
    import threading
    from paper_1603_09180_gb300 import thin
    srv = thin.Server(SERVE_BUDGET, max_slots=slots, queue_cap=queue)
    done_t, errors = {}, []
    lock = threading.Lock()

    def submit(img, lam):
        try:
            return srv.submit(img, lam)
        except thin.ThinError as e:
            if e.code == thin.THIN_EAGAIN:
                return None
            raise

    def collector(stop):
        while True:
            t = srv.wait_any(50)
            if t is None:
                if stop.is_set():
                    return
                continue
            td = time.perf_counter()
            ok, res, st, rc = srv.poll(t)
            with lock:
                if ok and rc == 0:
                    done_t[t] = td
                else:
                    errors.append(rc)

    stop = threading.Event()
    col = threading.Thread(target=collector, args=(stop,), daemon=True)
    col.start()

    def drain(n):
        t_lim = time.perf_counter() + 120
        while time.perf_counter() < t_lim:
            with lock:
                if len(done_t) + len(errors) >= n:
                    break
            time.sleep(0.002)
        stop.set()
        col.join()
        return dict(done_t)

    r = _drive(rate, seconds, pool, submit, drain)
    r["errors"] = len(errors)
    srv.close()
    return r


def serve_plain(pool, rate, seconds, queue, dev):
    """The plain path at the same arrivals: one worker, one image at a time (H2D, thin_run, D2H)."""
    import queue as qmod
    import threading
    from paper_1603_09180_gb300 import thin
    q = qmod.Queue(maxsize=queue)
    done_p, errors_p = {}, []
    nxt = [0]

    def worker():
        while True:
            item = q.get()
            if item is None:
                return
            tk, img, lam = item
            try:
                t = _to_dev(img, dev)
                thin.run(t, lam, stats=False)
                t.cpu()
                done_p[tk] = time.perf_counter()
            except Exception:
                errors_p.append(tk)

    wt = threading.Thread(target=worker, daemon=True)
    wt.start()

    def submit_p(img, lam):
        nxt[0] += 1
        try:
            q.put_nowait((nxt[0], img, lam))
            return nxt[0]
        except qmod.Full:
            return None

    def drain_p(n):
        t_lim = time.perf_counter() + 120
        while len(done_p) + len(errors_p) < n and time.perf_counter() < t_lim:
            time.sleep(0.002)
        q.put(None)
        wt.join(timeout=5)
        return dict(done_p)

    r = _drive(rate, seconds, pool, submit_p, drain_p)
    r["errors"] = len(errors_p)
    return r


def service_times_ms(pool, lams, dev):
    """Each pool image alone, end to end (H2D, thin_run, D2H), wall ms; after one warm-up pass."""
    import torch
    from paper_1603_09180_gb300 import thin
    out = []
    for rep in range(2):
        for img, lam in zip(pool, lams):
            t0 = time.perf_counter()
            t = _to_dev(img, dev)
            thin.run(t, lam, stats=False)
            t.cpu()
            torch.cuda.synchronize()
            if rep:
                out.append(1e3 * (time.perf_counter() - t0))
    return sorted(out)


def serve_closed(pool, n, slots, queue):
    """The mix's throughput with every request queued at once: n requests (the pool cycled, lambda from the
    trace), images/s from the first submit to the last completion.  Unlike a saturated open-loop run, whose
    rejections let the light images through while the large ones wait, every image of the mix counts."""
    from paper_1603_09180_gb300 import synth, thin
    _, spec = synth.serve_trace(1000.0, n)
    srv = thin.Server(SERVE_BUDGET, max_slots=slots, queue_cap=max(queue, n))
    t0 = time.perf_counter()
    done, k = 0, 0
    while done < n:
        while k < n:
            try:
                srv.submit(pool[k % len(pool)], spec[k][3])
                k += 1
            except thin.ThinError as e:
                if e.code != thin.THIN_EAGAIN:
                    raise
                break  # host staging full: take a result first
        t = srv.wait_any(60000)
        if t is None:
            raise RuntimeError("no request finished within 60 s")
        ok, _, _, rc = srv.poll(t)
        if not ok or rc != 0:
            raise RuntimeError("request failed: %d" % rc)
        done += 1
    secs = time.perf_counter() - t0
    srv.close()
    return {"requests": n, "seconds": round(secs, 3), "images_per_s": round(n / secs, 1)}


def serve_summary(pool, lams, dev, slots, queue, seconds):
    """Serving capacity (the whole mix queued at once), at saturation and at half of the capacity, with
    the single-image service time of the mix: the figures the default benchmark line carries."""
    svc = service_times_ms(pool, lams, dev)
    closed = serve_closed(pool, 4 * len(pool), slots, queue)
    sat = serve_served(pool, 20000.0, 2.0, slots, queue)
    cap = max(1.0, closed["images_per_s"])
    half = serve_served(pool, 0.5 * cap, max(seconds, min(15.0, 600.0 / (0.5 * cap))), slots, queue)
    p50svc = round(svc[len(svc) // 2], 2)
    return {"capacity_images_per_s": cap, "capacity_run": closed, "saturated": sat, "at_half_capacity": half,
            "single_image_service_ms": {"p50": p50svc, "p90": round(svc[int(0.9 * (len(svc) - 1))], 2),
                                        "max": round(svc[-1], 2)},
            "p50_over_service_p50_at_half": round(half["p50_ms"] / p50svc, 2) if half["p50_ms"] else None}


def run_serve(args):
    """Poisson arrivals through thin_serve_* against a plain one-image-at-a-time path."""
    import torch
    from paper_1603_09180_gb300 import thin
    specs, lams = serve_pool_specs(args.serve_pool)
    pool = _gen_pool(specs, host_cores())
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    thin.load()
    out = {"served": [], "plain": []}
    with ClockSampler(0) as clk:
        summ = serve_summary(pool, lams, dev, args.serve_slots, args.serve_queue, args.serve_seconds)
        cap = summ["capacity_images_per_s"]
        rates = [float(r) for r in args.serve_rates.split(",")] + [f * cap for f in (0.25, 0.5, 0.9)]
        for rate in sorted(rates):
            # long enough for about 2000 completions below capacity (at most 20 s)
            secs = max(args.serve_seconds, min(20.0, 2000.0 / min(rate, cap)))
            r = serve_served(pool, rate, secs, args.serve_slots, args.serve_queue)
            out["served"].append(r)
            print("served", json.dumps(r), file=sys.stderr, flush=True)
        plain_cap = serve_plain(pool, 20000.0, 2.0, args.serve_queue, dev)["steady_images_per_s"]
        for f in (0.5, 2.0):
            r = serve_plain(pool, f * max(1.0, plain_cap), args.serve_seconds, args.serve_queue, dev)
            r["fraction_of_plain_capacity"] = f
            out["plain"].append(r)
            print("plain", json.dumps(r), file=sys.stderr, flush=True)
    head = summ["at_half_capacity"]
    return {"metric": "served images/s and p99 latency (Poisson arrivals)", "value": summ["capacity_images_per_s"],
            "unit": "images/s", "n_gpus": 1, "higher_is_better": True, "dtype": "u8/u16", "data": "synthetic",
            "workload": "serve",
            "config": {"workload": "Poisson arrivals, sides log-uniform [128, 4096], u8/u16 1:1, lambda {0, 10} "
                                   "on pixel values as given, %d-image pool cycled" % args.serve_pool,
                       "budget_bytes": SERVE_BUDGET, "max_slots": args.serve_slots, "queue_cap": args.serve_queue},
            "p50_ms_at_half_capacity": head["p50_ms"], "p99_ms_at_half_capacity": head["p99_ms"],
            "summary": summ, "rates": out, "plain_capacity_images_per_s": plain_cap, "clocks": clk.summary()}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--kernel", default="auto", choices=["auto", "resident", "tiled", "naive"])
    ap.add_argument("--halo", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--images", type=int, default=N_IMAGES, help="images per batch (profiling runs use fewer)")
    ap.add_argument("--no-large", action="store_true", help="skip the large-image figures of the default line")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving figures of the default line")
    ap.add_argument("--workload", default="batch192", choices=["batch192", "large", "uneven", "serve"])
    ap.add_argument("--uneven-n", type=int, default=1024)
    ap.add_argument("--serve-rates", default="1000,2000,5000,10000,20000,50000")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--serve-queue", type=int, default=256)
    args = ap.parse_args(argv)
    globals()["N_IMAGES"] = args.images
    if args.warmup < 3 and args.impl == "native":
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload != "batch192" and args.impl == "native":
        line = {"large": run_large, "uneven": run_uneven, "serve": run_serve}[args.workload](args) if rank == 0 else None
    elif args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        line = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
