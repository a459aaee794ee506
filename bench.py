#!/usr/bin/env python
"""Throughput of the CTIS EM reconstruction on GB300.

One step = one full reconstruction of the workload (k EM iterations with the
per-iteration float64 statistics) from resident device inputs, through the
library's public API. Default workload: field stop 128x128, 64 wavelengths,
1024x1024 FPA, 5x5 diffraction orders, 3x3 spots (225 nonzeros per
calibration image), 100 iterations; synthetic seeded inputs.

Prints one JSON line on rank 0. With --impl reference the FP64 CPU oracle is
timed instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reconstruction iterations/s and voxel-updates/s vs plain FP32; % roofline"
SMS, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_GHZ / 1e3   # 80.5 TFLOP/s
L2_FLUSH_BYTES = 256 << 20



def schedule_name(sched):
    """A plan schedule ``(kind, value, skew)`` in words."""
    kind, v, skew = sched
    name = (f"balanced split, item overhead {v / 4:g} tasks" if kind == "split"
            else f"chunks of <= {v} tasks, longest first")
    return name + (f", CTA priority skew {skew / 1000:g}" if skew else "")

def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="realistic_128x128x64_fpa1024")
    ap.add_argument("--k", type=int, default=None, help="EM iterations per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and autograd forms")
    ap.add_argument("--schedule", default=None,
                    help="skip the autotuner and use these schedules, 'FWD,ADJ' with each "
                         "'chunk:TASKS:SKEW' or 'split:OVERHEAD_Q:SKEW' (SKEW in permille), "
                         "FWD optionally led by its tile shape ('32x16:chunk:64:0'), "
                         "e.g. a bench line's schedule.spec")
    ap.add_argument("--paper-table", default=None, metavar="OUT_JSON",
                    help="instead of the bench line: the paper's Table 1 grid (field stop "
                         "89x80, 2048x2048 FPA, w = 3, 24, 75, K = 10..3100) on a synthetic PSF, "
                         "gather and FFT-form reconstruction times beside the paper's P4000 "
                         "times; writes OUT_JSON and prints a one-line summary")
    ap.add_argument("--fma-peak", action="store_true",
                    help="instead of the bench line: the FP32 FMA-pipe microbenchmark alone "
                         "(one JSON line)")
    ap.add_argument("--crossover", default=None, metavar="OUT_JSON",
                    help="instead of the bench line: sweep the spot size on the realistic "
                         "geometry, time the gather and the FFT form per EM iteration, write "
                         "the table to OUT_JSON and print a one-line summary")
    return ap.parse_args()


def aggregate_over_ranks(total_ms, total_e2e, steps, k, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` replicas that each ran `steps` steps of
    k EM iterations: the job's time is the slowest rank's (max over ranks),
    its work all ranks' iterations. Returns (value, e2e value, job ms, job e2e
    ms); every rank gets the same numbers."""
    if dist is not None:
        import torch
        t = torch.tensor([total_ms, total_e2e], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, total_e2e = float(t[0]), float(t[1])
    iters = steps * k * world
    return iters / (total_ms / 1e3), iters / (total_e2e / 1e3), total_ms, total_e2e


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_median": statistics.median(power), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- helpers
def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("ctis_gather.cuh", "ctis_gather_fwd.cu", "ctis_gather_adj.cu", "ctis_gather.cu",
                 "ctis_internal.h"):
        with open(os.path.join(ROOT, "paper_2006_01573_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str, units_scale: float = 1.0):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    when the kernel sources changed since those counters were taken or they
    were taken on another workload."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        return None
    if data.get("source_hash") != kernel_source_hash() or data.get("workload") != workload:
        return None
    entry = data.get("kernels", {}).get(kernel)
    return None if entry is None else entry["dram_bytes_per_launch"] * units_scale


def measure_fma_peak():
    """The FP32 FMA-pipe microbenchmark (ctis_fma_peak): TFLOP/s with scalar
    FFMA and with FFMA2 pairs, at 64 warps per SM and at the projectors' 16."""
    from paper_2006_01573_gb300 import fma_peak
    out = {}
    for packed in (False, True):
        for bps, thr in ((8, 256), (4, 128)):
            key = f"{'ffma2' if packed else 'ffma'}_{bps * thr // 32}_warps_per_sm"
            out[key] = fma_peak(packed=packed, blocks_per_sm=bps, threads=thr)
    out["best_tflops"] = max(out.values())
    out["nominal_tflops"] = FP32_PEAK_TFLOPS
    out["kernel"] = "ctis_fma_peak: 8 independent chains x 4 FMAs per iteration per thread"
    return out


def problem(wl, seed):
    import numpy as np  # noqa: F401
    import synth
    return synth.make_psf(wl), synth.make_scene(wl, seed)


# --------------------------------------------------------------------------- oracle
_ORACLE_CACHE = {}


def oracle_problem(wl):
    """The FP64 oracle's full-size problem: its sparse H (every wavelength
    block, Eq. 3 partition, scipy CSR) and the Poisson counts of the scene as
    the oracle itself images it (nothing from the GPU path). Built once per
    process; returns (H, h, g, seconds to build)."""
    if wl.name not in _ORACLE_CACHE:
        import numpy as np

        import oracle as O
        import synth
        t0 = time.perf_counter()
        geom = O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
        H = O.BlockH(geom, O.merge_psf(geom, synth.make_psf(wl)))
        g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
        _ORACLE_CACHE[wl.name] = (H, H.h(), np.asarray(g, dtype=np.float64).ravel(),
                                  time.perf_counter() - t0)
    return _ORACLE_CACHE[wl.name]


def oracle_iterations(wl, n_iter: int):
    """n_iter EM iterations (Eq. 2) of the FP64 oracle on the full workload
    from all ones, each timed on its own. Returns the list of seconds."""
    import numpy as np

    import oracle as O
    H, h, g, _ = oracle_problem(wl)
    f = np.ones(H.geom.m)
    secs = []
    for _ in range(n_iter):
        t0 = time.perf_counter()
        f = O.em_update(f, H.adjoint(O.ratio(g, H.forward(f))), h)
        secs.append(time.perf_counter() - t0)
    return secs


def oracle_reconstruction(wl, k: int):
    """The benchmarked reconstruction done by the FP64 oracle: k EM updates
    (Eq. 2) of the full workload from ones on the oracle's own measurement,
    each timed. Returns (f, seconds per update, seconds to build H)."""
    import numpy as np

    import oracle as O
    H, h, g, build_s = oracle_problem(wl)
    f = np.ones(H.geom.m)
    secs = []
    for _ in range(k):
        t0 = time.perf_counter()
        f = O.em_update(f, H.adjoint(O.ratio(g, H.forward(f))), h)
        secs.append(time.perf_counter() - t0)
    return f, secs, build_s


def accuracy_vs_oracle(wl, k, f_ref):
    """The GPU reconstruction of the benchmarked workload against the FP64
    oracle's (same input: the oracle's measurement), for the float32 plan and
    the bfloat16-storage plan, both autotuned as in the timed runs: max
    floored-relative error (floor 1e-6 of the maximum) and relative L2 over
    every voxel after k updates from ones."""
    import numpy as np
    import torch

    import synth
    from paper_2006_01573_gb300 import Plan
    _, _, g, _ = oracle_problem(wl)
    gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma).astype(np.float32)).cuda()
    out = {}
    for dtype in ("f32", "bf16"):
        plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl), dtype=dtype)
        plan.autotune(gt)
        f, _ = plan.reconstruct(gt, k, init="ones")
        plan.check()
        a = f.double().cpu().numpy().ravel()
        plan.close()
        floor = 1e-6 * np.abs(f_ref).max()
        out[dtype] = {"max_floored_rel": float(np.max(np.abs(a - f_ref) / np.maximum(np.abs(f_ref), floor))),
                      "rel_l2": float(np.linalg.norm(a - f_ref) / np.linalg.norm(f_ref))}
    out["reference"] = (f"float64 oracle, {k} EM updates from ones on every voxel of the "
                        f"{wl.name} workload, the oracle's own noisy measurement")
    return out


def run_reference(args, wl, k):
    """The reference arm: the FP64 oracle as it stands, on the host cores.
    One step is ONE EM iteration of the full workload (the oracle runs about
    two per second, so a step of the workload's k iterations would not fit
    the run); steps and ms_per_step describe exactly those iterations."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    _, _, _, build_s = oracle_problem(wl)
    oracle_iterations(wl, args.warmup)
    secs = oracle_iterations(wl, args.steps)
    value = len(secs) / sum(secs)
    desc = (f"{wl.name}: {len(secs)} timed full-size EM iterations of the float64 oracle "
            f"(scipy CSR sparse H of every wavelength block, 1 thread) after {args.warmup} "
            f"untimed ones; H built once in {build_s:.1f} s, not timed")
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(secs) / len(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded PSF, scene, Poisson noise)",
        "step": "one EM iteration of the full workload (the workload's k iterations would take "
                f"{k * sum(secs) / len(secs):.0f} s per step)",
        "config": bench_config(wl, k, world),
        "voxel_updates_per_s": value * wl.m,
        "cpu_baseline": {"value": value, "unit": "it/s", "cores": 1, "kind": "oracle",
                         "sample": desc, "host_cpus": os.cpu_count()},
        "e2e": {"value": value, "unit": "it/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_config(wl, k, world):
    """The bench line's config (both arms print the same keys)."""
    return {"workload": wl.name, "k": k, "a": wl.a, "alpha": wl.alpha, "w": wl.w,
            "gamma": wl.gamma, "xi": wl.xi, "orders": f"{wl.orders}x{wl.orders}",
            "spot": f"{wl.spot}x{wl.spot}", "nnz_per_image": wl.nnz_per_image,
            "voxels": wl.m, "parallelism": f"replicas x{world}",
            "l2": "flushed between timed steps (256 MiB write)",
            "stats": "float64 flux/loglik/resid per iteration"}


# --------------------------------------------------------------------------- ours
def run_ours(args, wl, k):
    import numpy as np
    import torch

    import synth
    from paper_2006_01573_gb300 import Plan

    rank, world, local = dist_env()
    # the batched form's oracle frames run in spawned workers meanwhile
    oracle_job = (start_batched_oracle() if world == 1 and not args.no_forms and
                  not args.no_cpu_baseline else None)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    seed = wl.seed + rank
    psf = synth.make_psf(wl)
    f_true = synth.make_scene(wl, seed)
    specs = args.schedule.split(",") if args.schedule else None
    tile = "32x32"
    if specs and specs[0].count(":") == 3:        # the forward's spec led by its tile shape
        tile, specs[0] = specs[0].split(":", 1)
    plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, forward_tile=tile)
    hf = plan.forward(torch.from_numpy(f_true).to(dev))
    g_host, _ = synth.make_measurement(hf.cpu().numpy(), wl.peak, seed)
    g = torch.from_numpy(g_host).to(dev)
    if specs:                                     # a given schedule (e.g. to profile one)
        for forward, spec in zip((True, False), specs):
            kind, value, skew = spec.split(":")
            plan.set_schedule(forward, (kind, int(value), int(skew)))
        tuned = plan.schedules()
    else:
        tuned = plan.autotune(g)                  # schedule autotuner (plan setup)
    info = plan.info()
    f = torch.empty((wl.w, wl.alpha, wl.a), device=dev, dtype=torch.float32)
    stats = torch.empty((k + 1, 4), device=dev, dtype=torch.float64)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()
    plan.set_profiling(False)   # the value's steps run without event nodes in the graph

    def step():
        plan.reconstruct(g, k, f=f, init="ones", stats=stats)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall0 = time.perf_counter()
    step_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))                      # evict L2 between timed steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    # Per-kernel durations: the same steps again with a CUDA event pair around
    # every projector launch (event-record nodes of the reconstruction graph,
    # on the launching stream). Those nodes add ~15 us per iteration to the
    # step, so the value above comes from steps without them.
    plan.set_profiling(True)
    step()
    torch.cuda.synchronize()
    fwd_ms, adj_ms, n_fwd, n_adj, prof_ms = 0.0, 0.0, 0, 0, 0.0
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        prof_ms += e0.elapsed_time(e1)
        kt = plan.kernel_times()
        fwd_ms += kt["forward"][0]
        n_fwd += kt["forward"][1]
        adj_ms += kt["adjoint"][0]
        n_adj += kt["adjoint"][1]
    plan.set_profiling(False)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    plan.check()

    # ---- end to end through the public API from pinned host buffers
    g_pin = torch.from_numpy(g_host).pin_memory()
    f_pin = torch.empty(f.shape, dtype=f.dtype).pin_memory()
    st_pin = torch.empty(stats.shape, dtype=stats.dtype).pin_memory()
    g_dev = torch.empty_like(g)
    f_dev = torch.empty_like(f)

    def e2e_step():
        g_dev.copy_(g_pin, non_blocking=True)
        plan.reconstruct(g_dev, k, f=f_dev, init="ones", stats=stats)
        f_pin.copy_(f_dev, non_blocking=True)
        st_pin.copy_(stats, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))

    value, e2e_value, total_ms, total_e2e = aggregate_over_ranks(
        sum(step_ms), sum(e2e_ms), args.steps, k, world, dist, dev)

    # ---- roofline of the dominant kernel: its average device time per launch
    # over back-to-back launches of that kernel alone (no event between the
    # launches), L2 flushed first; the event pairs around every launch of the
    # profiled steps above give the kernels' shares of a step
    nnz_h = info["nnz"] * wl.a * wl.alpha          # nonzeros of H = FMAs per projection
    flops = 2.0 * nnz_h
    reps = 50
    flush.fill_(0.5)
    b2b = plan.time_launches(g, reps)
    b2b_ms = {"forward": b2b[0], "adjoint": b2b[1]}
    kernels = {"forward": (fwd_ms, n_fwd), "adjoint": (adj_ms, n_adj)}
    dom = max(b2b_ms, key=lambda n: b2b_ms[n])
    avg_ms = b2b_ms[dom]
    achieved = flops / (avg_ms * 1e-3) / 1e12
    per_kernel = {n: {"launches_profiled": c,
                      "avg_us_back_to_back": 1e3 * b2b_ms[n],
                      "tflops_back_to_back": flops / (b2b_ms[n] * 1e-3) / 1e12,
                      "avg_us_with_event_nodes": 1e3 * t / max(1, c),
                      "share_of_step": t / prof_ms if prof_ms else None}
                  for n, (t, c) in kernels.items()}
    fma = measure_fma_peak() if rank == 0 else None
    if world > 1:
        per_kernel = {n: v for n, v in per_kernel.items()}   # rank 0's view

    if rank != 0:
        plan.close()
        if dist:
            dist.destroy_process_group()
        return

    line = {
        "metric": METRIC, "value": value, "unit": "it/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded PSF, scene, Poisson noise)",
        "config": bench_config(wl, k, world),
        # the work schedule the plan ran (kept out of config, which both arms
        # print identically)
        "schedule": {"forward": f"{plan.forward_tile()} tiles, " + schedule_name(tuned[0]),
                     "adjoint": schedule_name(tuned[1]),
                     "spec": plan.forward_tile() + ":" +
                             ",".join(f"{k}:{v}:{sk}" for k, v, sk in tuned),
                     "chosen_by": "--schedule" if args.schedule else "ctis_plan_autotune"},
        "voxel_updates_per_s": value * wl.m,
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": ncu_traffic(dom, wl.name),
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 FLOP/FMA x 2070 MHz (max SM clock)",
                     "measured_fma_peak": fma["best_tflops"],
                     "frac_of_measured_fma_peak": achieved / fma["best_tflops"],
                     "timing": f"CUDA events around {reps} back-to-back EM launches of the kernel "
                               "(ctis_plan_time_launches, no event between launches), after the "
                               "timed region on the same workload",
                     "algorithmic_flops_per_launch": flops},
        "fma_peak": fma,
        "kernels": per_kernel,
        "e2e": {"value": e2e_value, "unit": "it/s",
                "h2d_bytes_per_step": g_pin.numel() * 4,
                "d2h_bytes_per_step": f_pin.numel() * 4 + st_pin.numel() * 8},
        # per step: f scatter, k + 1 forwards (the last for the statistics), k adjoints,
        # the last forward's statistics reduction, f out
        "gpu_launches": args.steps * (2 * k + 4),
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    line["forms"] = {"bf16": bf16_form(args, wl, k, psf, g, f, flush, stream, value),
                     "solvers": solver_forms(args, wl, k, plan, g, flush, stream, value)}
    if world == 1 and not args.no_forms:
        line["forms"]["sharded"] = sharded_form(args, wl, k, plan, g, flush, stream, value)
        line["forms"]["fft"] = fft_form(args, wl, psf, g, f, flush, stream, value)
        line["forms"]["batched"] = batched_form(args, flush, stream, oracle_job=oracle_job)
        line["forms"]["large"] = large_form(args, flush, stream, fma)
        line["forms"]["autograd"] = autograd_form(args, flush, stream)
    plan.close()
    if world == 1 and not args.no_cpu_baseline:
        f_ref, secs, build_s = oracle_reconstruction(wl, k)
        v = len(secs) / sum(secs)
        desc = (f"{wl.name}: the whole benchmarked reconstruction, {len(secs)} full-size EM "
                f"updates of the float64 oracle (scipy CSR sparse H of every wavelength block, "
                f"1 thread) in {sum(secs):.1f} s, from ones; H built once in {build_s:.1f} s, "
                f"not timed")
        line["cpu_baseline"] = {"value": v, "unit": "it/s", "cores": 1, "kind": "oracle",
                                "sample": desc, "host_cpus": os.cpu_count()}
        line["accuracy_vs_fp64_oracle"] = accuracy_vs_oracle(wl, k, f_ref)
        if "forms" in line and "bf16" in line["forms"]:
            line["forms"]["bf16"]["vs_fp64_oracle_after_k"] = line["accuracy_vs_fp64_oracle"]["bf16"]
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def bf16_form(args, wl, k, psf, g, f32_result, flush, stream, f32_value):
    """The bfloat16 storage form (datacube and PSF values in bfloat16, float32
    sums) on the same workload and g: its iterations/s, the ratio to the plain
    float32 path, and the relative L2 distance of its reconstruction from the
    float32 one after k iterations."""
    import torch
    from paper_2006_01573_gb300 import Plan
    plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype="bf16")
    plan.autotune(g)
    fb = torch.empty(f32_result.shape, device=g.device, dtype=torch.bfloat16)
    stats = torch.empty((k + 1, 4), device=g.device, dtype=torch.float64)
    for _ in range(max(1, args.warmup)):
        plan.reconstruct(g, k, f=fb, init="ones", stats=stats)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    total = 0.0
    for i in range(steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.reconstruct(g, k, f=fb, init="ones", stats=stats)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    plan.check()
    value = steps * k / (total / 1e3)
    a = fb.double()
    b = f32_result.double()
    err = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    plan.close()
    return {"value": value, "unit": "it/s", "steps": steps, "vs_f32": value / f32_value,
            "rel_l2_vs_f32_after_k": err, "dtype": "bf16 storage, f32 accumulate"}


def solver_forms(args, wl, k, plan, g, flush, stream, em_value):
    """SART and SMART (ctis_reconstruct_solver, relaxation 1) on the same plan,
    workload and g, with the per-iteration statistics: their iterations/s and
    the ratio to EM's (the same two launches per iteration, other epilogue
    rules)."""
    import torch
    f = torch.empty((wl.w, wl.alpha, wl.a), device=g.device)
    stats = torch.empty((k + 1, 4), device=g.device, dtype=torch.float64)
    out = {}
    for solver in ("sart", "smart"):
        run = lambda: plan.reconstruct(g, k, f=f, init="ones", stats=stats, solver=solver)
        for _ in range(max(1, args.warmup)):
            run()
        torch.cuda.synchronize()
        steps = max(1, min(args.steps, 5))
        total = _timed_steps(run, steps, flush, stream)
        plan.check()
        value = steps * k / (total / 1e3)
        out[solver] = {"value": value, "unit": "it/s", "steps": steps, "vs_em": value / em_value,
                       "relax": 1.0}
    return out


def sharded_form(args, wl, k, plan, g, flush, stream, em_value):
    """The wavelength-sharded EM path (ctis_reconstruct_sharded) with the
    whole datacube as its one slice and no reduction, on the same plan and g:
    its iterations/s against the graph-captured EM. One GPU: this measures
    the path's own cost (its host loop of launches, the partial image and the
    separate ratio kernel in place of the fused one), not a scaling."""
    import torch
    f = torch.empty((wl.w, wl.alpha, wl.a), device=g.device)
    run = lambda: plan.reconstruct_sharded(g, k, f=f, init="ones", stats=True)
    for _ in range(max(1, args.warmup)):
        run()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3))
    total = _timed_steps(run, steps, flush, stream)
    plan.check()
    value = steps * k / (total / 1e3)
    return {"value": value, "unit": "it/s", "steps": steps, "slices": 1, "vs_em_graph": value / em_value,
            "exchange_bytes_per_iteration_per_rank": 4 * wl.gamma * wl.xi,
            "note": "one slice, no reduction; multi-GPU scaling unmeasured (one GPU)"}


def fft_form(args, wl, psf, g, f32_result, flush, stream, f32_value, k=33):
    """The paper's own (WBH) form of the projectors, on the same workload and
    g: k EM updates (33, as the paper's validation) with cuFFT transforms of
    length n and this project's spectral multiply-accumulate and index maps
    (Eqs. 11, 13, 14, 17). Its iterations/s, the ratio to the gather path, and
    its distance from the gather reconstruction after k iterations (both from
    ones): relative L2 and the paper's average relative pixel error (Sec. 4,
    over the voxels above 1e-6 of the maximum)."""
    import torch
    from paper_2006_01573_gb300 import Plan
    plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf)
    f = torch.empty(f32_result.shape, device=g.device)
    for _ in range(max(1, args.warmup)):
        plan.fft_reconstruct(g, k, f=f.fill_(1.0))
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3))
    total = _timed_steps(lambda: plan.fft_reconstruct(g, k, f=f.fill_(1.0)), steps, flush, stream)
    ref, _ = plan.reconstruct(g, k, init="ones")
    plan.check()
    a, b = f.double(), ref.double()
    err = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    on = b > 1e-6 * b.max()
    avg_rel = float(((a[on] - b[on]).abs() / b[on]).mean())
    plan.close()
    value = steps * k / (total / 1e3)
    # HBM bytes of one iteration if every pass reads and writes its operands
    # once: the w-batched R2C and C2R (4 n w real, 8 beta w complex each way),
    # the spectral multiply-accumulate (X and the PSF spectra D in, S out) and
    # its adjoint expansion (S and D in, X out); the n- and m-sized passes
    # (embedding, ratio, single transforms, crop, update) add < 1%
    n, w = wl.gamma * wl.xi, wl.w
    beta = n // 2 + 1
    nbytes = 2 * (4 * n * w + 8 * beta * w) + 2 * (16 * beta * w + 8 * beta)
    hbm = measured_hbm_gbs()
    return {"value": value, "unit": "it/s", "k": k, "steps": steps, "vs_gather": value / f32_value,
            "rel_l2_vs_gather_after_k": err, "avg_rel_pixel_err_vs_gather_after_k": avg_rel,
            "roofline": {"bound": "hbm", "algorithmic_bytes_per_iteration": nbytes,
                         "achieved_gbs": nbytes * value / 1e9, "peak_gbs": hbm,
                         "frac": nbytes * value / 1e9 / hbm,
                         "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"},
            "form": "cuFFT R2C/C2R of length n per wavelength + spectral MAC (float32)"}


def measured_hbm_gbs():
    """The machine's measured HBM copy bandwidth in GB/s (MEASURED_PEAKS.json),
    else the earlier GB300 measurement of 6 800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def _timed_steps(fn, steps, flush, stream):
    import torch
    total = 0.0
    for i in range(steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total


def _oracle_frame(args):
    """One sampled frame of the batched form, done by the FP64 oracle (run in
    a spawned worker process): the frame's scene imaged by the oracle, its
    Poisson counts (seed 1000 + i), and k EM updates from ones."""
    name, i, k = args
    import numpy as np

    import oracle as O
    import synth
    wl = synth.WORKLOADS[name]
    geom = O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    H = O.build_H(geom, synth.make_psf(wl))
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl, 1000 + (1000 + i) % 8).ravel()),
                                  wl.peak, 1000 + i)
    f, _ = O.mlem(H, g, k)
    return i, np.asarray(g, dtype=np.float32), f


# frames of the 256-frame mix whose error against the FP64 oracle is reported
# (plan A when i % 4 != 3, plan B otherwise)
BATCH_SAMPLE_FRAMES = (0, 1, 2, 4, 3, 7)


def start_batched_oracle(k=100):
    """Starts the oracle's sampled frames in a spawned process pool (one
    worker per frame); returns (pool, async result)."""
    import multiprocessing as mp
    import synth
    jobs = [((synth.MODEL_B if i % 4 == 3 else synth.MODEL_A).name, i, k) for i in BATCH_SAMPLE_FRAMES]
    pool = mp.get_context("spawn").Pool(len(jobs))
    return pool, pool.map_async(_oracle_frame, jobs)


def batched_form(args, flush, stream, nframes=256, k=100, oracle_job=None):
    """The batched form: 256 frames, 3:1 of the 64x64x32 -> 512^2 and the
    128x128x64 -> 1024^2 geometry, k EM iterations with per-frame statistics,
    one ctis_reconstruct_batched call per step, timed with float32 and with
    bfloat16 storage. Frame i: plan B when i % 4 == 3, else A; scene
    (1000 + i) % 8 of its geometry (8 scenes each, cycled), Poisson counts of
    H f scaled to the workload's peak drawn on the GPU with seed 1000 + i.
    With oracle_job (start_batched_oracle): per-frame error against the FP64
    oracle on the sampled frames, whose inputs are then the oracle's own
    measurements (frames are bit-identical to their single-frame runs in any
    batch, so the sample's errors are those of the same frames in the
    256-frame batch)."""
    import numpy as np
    import torch
    import synth
    from paper_2006_01573_gb300 import Plan, reconstruct_batched
    wls = [synth.MODEL_A, synth.MODEL_B]
    plan_idx = [1 if i % 4 == 3 else 0 for i in range(nframes)]
    out = {"frames": nframes, "mix": "192 x 64x64x32->512^2 + 64 x 128x128x64->1024^2", "k": k}
    gs = None
    for dtype in ("f32", "bf16"):
        plans = [Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl), dtype=dtype)
                 for wl in wls]
        if gs is None:
            scenes = [[torch.from_numpy(synth.make_scene(wl, 1000 + j)).cuda() for j in range(8)]
                      for wl in wls]
            gs = []
            for i, p in enumerate(plan_idx):
                hf = plans[p].forward(scenes[p][(1000 + i) % 8].to(plans[p]._f_dtype()))
                gen = torch.Generator(device="cuda").manual_seed(1000 + i)
                gs.append(torch.poisson(hf * (wls[p].peak / hf.max()), generator=gen))
            del scenes
        for p in range(len(plans)):                   # tune each plan on one of its frames
            plans[p].autotune(gs[plan_idx.index(p)])
        tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
        fs = [torch.empty((wls[p].w, wls[p].alpha, wls[p].a), device="cuda", dtype=tdt)
              for p in plan_idx]
        stats = torch.empty((nframes, k + 1, 4), device="cuda", dtype=torch.float64)

        def step():
            reconstruct_batched(plans, plan_idx, gs, k, fs=fs, init="ones", stats=stats)

        for _ in range(max(1, args.warmup)):
            step()
        torch.cuda.synchronize()
        steps = max(1, min(args.steps, 3))
        total = _timed_steps(step, steps, flush, stream)
        for p in plans:
            p.check()
        voxels = sum(wls[p].m for p in plan_idx)
        secs = total / 1e3
        out[dtype] = {"steps": steps, "ms_per_step": total / steps,
                      "frame_iterations_per_s": steps * nframes * k / secs,
                      "voxel_updates_per_s": steps * voxels * k / secs}
        if oracle_job is not None:
            res = oracle_job[1].get(timeout=900)
            sub_idx = [plan_idx[i] for i, _, _ in res]
            sub_g = [torch.from_numpy(g.reshape(wls[plan_idx[i]].xi, wls[plan_idx[i]].gamma)).cuda()
                     for i, g, _ in res]
            sub_f, _ = reconstruct_batched(plans, sub_idx, sub_g, k, init="ones")
            per = {}
            for (i, _, f_ref), f in zip(res, sub_f):
                a = f.double().cpu().numpy().ravel()
                floor = 1e-6 * np.abs(f_ref).max()
                per[str(i)] = {"plan": "B" if plan_idx[i] else "A",
                               "max_floored_rel": float(np.max(np.abs(a - f_ref) /
                                                               np.maximum(np.abs(f_ref), floor))),
                               "rel_l2": float(np.linalg.norm(a - f_ref) / np.linalg.norm(f_ref))}
            out[dtype]["vs_fp64_oracle_sampled_frames"] = per
        for p in plans:
            p.close()
        del fs, stats
    out["bf16_vs_f32"] = out["bf16"]["frame_iterations_per_s"] / out["f32"]["frame_iterations_per_s"]
    # per plan: g gather, f scatter, k + 1 forwards, k adjoints, f out, the last
    # forward's statistics reduction, statistics rows
    out["launches_per_step"] = len(wls) * (2 * k + 6)
    out["data"] = ("8 scenes per geometry cycled, per-frame Poisson noise on the GPU; error "
                   "sample: frames " + ", ".join(map(str, BATCH_SAMPLE_FRAMES)) +
                   " with the oracle's own measurements, the oracle in a spawned process pool")
    if oracle_job is not None:
        oracle_job[0].close()
    return out


def large_form(args, flush, stream, fma=None):
    """The large workload (256x256x128 cube, 2048x2048 FPA, 5x5 orders of
    5x5 spots: 625 nonzeros per image, K = 5 clusters), k = 50 EM iterations
    with statistics per step: iterations/s, voxel-updates/s and the FP32
    FLOP rate of the two projections; then each projector's EM launch alone
    (CUDA events around back-to-back launches) against the FP32 peak."""
    import torch
    import synth
    from paper_2006_01573_gb300 import Plan
    wl = synth.LARGE
    k = wl.k
    psf = synth.make_psf(wl)
    plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf)
    hf = plan.forward(torch.from_numpy(synth.make_scene(wl)).cuda())
    g = torch.poisson(hf * (wl.peak / hf.max()), generator=torch.Generator(device="cuda").manual_seed(wl.seed))
    tuned = plan.autotune(g)
    f = torch.empty((wl.w, wl.alpha, wl.a), device="cuda")
    stats = torch.empty((k + 1, 4), device="cuda", dtype=torch.float64)
    run = lambda: plan.reconstruct(g, k, f=f, init="ones", stats=stats)
    for _ in range(max(1, args.warmup)):
        run()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 3))
    total = _timed_steps(run, steps, flush, stream)
    plan.check()
    info = plan.info()
    reps = 20
    fwd_ms, adj_ms = plan.time_launches(g, reps)
    tile = plan.forward_tile()
    plan.close()
    value = steps * k / (total / 1e3)
    flops = 2 * 2 * int(info["nnz"]) * wl.a * wl.alpha   # two projections, 2 FLOP per FMA
    one = flops / 2                                       # one projection
    kernels = {}
    for name, ms in (("forward", fwd_ms), ("adjoint", adj_ms)):
        tf = one / (ms * 1e-3) / 1e12
        kernels[name] = {"avg_us_back_to_back": ms * 1e3, "tflops": tf,
                         "frac_of_nominal_peak": tf / FP32_PEAK_TFLOPS}
        if fma:
            kernels[name]["frac_of_measured_fma_peak"] = tf / fma["best_tflops"]
    return {"workload": wl.name, "k": k, "steps": steps, "value": value, "unit": "it/s",
            "voxel_updates_per_s": value * wl.m, "tflops_two_projections": value * flops / 1e12,
            "cluster_k": int(info["cluster_k"]), "forward_tile": tile,
            "schedule_spec": tile + ":" + ",".join(f"{kd}:{v}:{sk}" for kd, v, sk in tuned),
            "kernels": kernels,
            "kernel_timing": f"CUDA events around {reps} back-to-back EM launches of each kernel "
                             "(ctis_plan_time_launches), after the timed steps",
            "data": "seeded scene, Poisson counts of the GPU image drawn on the GPU"}


def autograd_form(args, flush, stream, k=10):
    """The autograd form: Poisson NLL after 10 unrolled EM updates of the
    realistic workload and its gradient with respect to every PSF value
    (checkpointed iterates, native backward pass), one call per step."""
    import torch
    import synth
    from paper_2006_01573_gb300 import Plan
    wl = synth.AUTOGRAD
    plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl))
    hf = plan.forward(torch.from_numpy(synth.make_scene(wl)).cuda())
    g_host, _ = synth.make_measurement(hf.cpu().numpy(), wl.peak, wl.seed)
    g = torch.from_numpy(g_host).cuda()
    plan.autotune(g)

    def step():
        plan.unrolled_nll_grad(g, k)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    total = _timed_steps(step, steps, flush, stream)
    plan.check()
    info = plan.info()
    plan.close()
    return {"workload": wl.name, "k_unrolled": k, "steps": steps, "ms_per_step": total / steps,
            "value_and_grad_per_s": steps / (total / 1e3),
            "unrolled_iterations_per_s": steps * k / (total / 1e3),
            "grad_entries": int(info["nnz"])}


# Table 1 of the paper: WBH + EM + P4000 reconstruction times in seconds, by
# (w, K) (Quadro P4000, FP32 FFT form; context only: other hardware, and the
# paper's calibration matrix is not available, so the PSF here is synthetic)
PAPER_TABLE1_P4000_S = {
    (75, 3100): 467.2, (75, 50): 7.5, (75, 33): 5.0, (75, 25): 3.8, (75, 10): 1.5,
    (24, 3100): 153.2, (24, 50): 2.5, (24, 33): 1.6, (24, 25): 1.2, (24, 10): 0.5,
    (3, 3100): 24.0, (3, 50): 0.4, (3, 33): 0.3, (3, 25): 0.2, (3, 10): 0.08,
}


def run_paper_table(args, fft_max_k=33):
    """The paper's Table 1 grid on GB300: its field stop (89x80), FPA
    (2048x2048) and wavelength counts (3, 24, 75), with a synthetic CTIS PSF
    (5x5 orders, pitch 360, dispersion 2 px per wavelength, 3x3 spots: 225
    nonzeros per image) standing in for the unavailable calibration matrix.
    Per (w, K): seconds for K EM updates with statistics through the gather
    path (autotuned; one timed run after a warm-up, L2 flushed), and through
    the FFT form for K <= fft_max_k, beside the paper's P4000 time."""
    import torch
    import synth
    from paper_2006_01573_gb300 import Plan
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    rows = []
    for w in (3, 24, 75):
        wl = synth.Workload(f"paper_89x80x{w}_fpa2048", 89, 80, w, 2048, 2048, 5, 360.0, 2.0, 3,
                            0.8, "segmentation", 4000.0, 10)
        psf = synth.make_psf(wl)
        plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf)
        hf = plan.forward(torch.from_numpy(synth.make_scene(wl)).cuda())
        gen = torch.Generator(device="cuda").manual_seed(wl.seed)
        g = torch.poisson(hf * (wl.peak / hf.max()), generator=gen)
        plan.autotune(g)
        f = torch.empty((wl.w, wl.alpha, wl.a), device="cuda")
        ff = torch.empty_like(f)
        for K in (10, 25, 33, 50, 3100):
            st = torch.empty((K + 1, 4), device="cuda", dtype=torch.float64)
            run = lambda: plan.reconstruct(g, K, f=f, init="ones", stats=st)
            run()
            torch.cuda.synchronize()
            t_g = _timed_steps(run, 1, flush, stream) / 1e3
            row = {"w": w, "K": K, "gather_s": t_g, "gather_it_per_s": K / t_g,
                   "paper_p4000_s": PAPER_TABLE1_P4000_S[(w, K)]}
            if K <= fft_max_k:
                fft = lambda: plan.fft_reconstruct(g, K, f=ff.fill_(1.0))
                fft()
                torch.cuda.synchronize()
                row["fft_s"] = _timed_steps(fft, 1, flush, stream) / 1e3
            rows.append(row)
        plan.check()
        plan.close()
        torch.cuda.empty_cache()
    out = {"geometry": "field stop 89x80, FPA 2048x2048 (the paper's); synthetic PSF: 5x5 orders, "
                       "pitch 360, dispersion 2, 3x3 spots (225 nonzeros per image)",
           "paper": "Table 1, WBH + EM on a Quadro P4000 (FP32 FFT form), context only",
           "rows": rows}
    with open(args.paper_table, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({"points": [(r["w"], r["K"], round(r["gather_s"], 4), r.get("fft_s") and
                                  round(r["fft_s"], 3), r["paper_p4000_s"]) for r in rows]}),
          flush=True)


CROSSOVER_SPOTS = (3, 5, 7, 9, 11, 13, 15, 17, 21)


def run_crossover(args, spots=CROSSOVER_SPOTS, k_gather=20, k_fft=5):
    """Gather vs the paper's FFT form as the PSF densifies: the realistic
    geometry (128x128x64 -> 1024^2, 5x5 orders) with square spots of side S
    (S^2 nonzeros per order, Gaussian sigma 0.8 S / 3, so 25 S^2 per
    calibration image). Per S: microseconds per EM iteration of each form
    (gather with its float64 statistics, autotuned; FFT without), L2
    flushed between timed runs, and the relative L2 distance of the two
    iterates after k_fft iterations. The gather's work grows with the
    nonzeros, the FFT form's does not; the crossover is where the two
    times meet, interpolated linearly in nnz between the bracketing sizes."""
    import torch
    import synth
    from paper_2006_01573_gb300 import Plan
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    steps = max(1, min(args.steps, 3))
    rows = []
    for S in spots:
        wl = synth.REALISTIC.with_(name=f"realistic_spot{S}", spot=S, sigma=0.8 * S / 3)
        psf = synth.make_psf(wl)
        plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf)
        hf = plan.forward(torch.from_numpy(synth.make_scene(wl)).cuda())
        g_host, _ = synth.make_measurement(hf.cpu().numpy(), wl.peak, wl.seed)
        g = torch.from_numpy(g_host).cuda()
        plan.autotune(g)
        f = torch.empty((wl.w, wl.alpha, wl.a), device="cuda")
        st = torch.empty((k_gather + 1, 4), device="cuda", dtype=torch.float64)
        gather = lambda: plan.reconstruct(g, k_gather, f=f, init="ones", stats=st)
        ff = torch.empty_like(f)
        fft = lambda: plan.fft_reconstruct(g, k_fft, f=ff.fill_(1.0))
        for _ in range(max(1, args.warmup)):
            gather()
            fft()
        torch.cuda.synchronize()
        t_g = _timed_steps(gather, steps, flush, stream) / steps / k_gather * 1e3
        t_f = _timed_steps(fft, steps, flush, stream) / steps / k_fft * 1e3
        ref, _ = plan.reconstruct(g, k_fft, init="ones")
        plan.check()
        err = float(torch.linalg.vector_norm(ff.double() - ref.double()) /
                    torch.linalg.vector_norm(ref.double()))
        info = plan.info()
        rows.append({"spot": S, "nnz_per_image": int(info["nnz"]) // wl.w,
                     "cluster_k": int(info["cluster_k"]), "gather_us_per_it": t_g,
                     "fft_us_per_it": t_f, "fft_over_gather": t_f / t_g,
                     "rel_l2_fft_vs_gather_after_k": err})
        plan.close()
        del f, ff, g, hf
        torch.cuda.empty_cache()
    cross = None
    for a, b in zip(rows, rows[1:]):
        da = a["gather_us_per_it"] - a["fft_us_per_it"]
        db = b["gather_us_per_it"] - b["fft_us_per_it"]
        if da <= 0 < db:
            t = -da / (db - da)
            cross = a["nnz_per_image"] + t * (b["nnz_per_image"] - a["nnz_per_image"])
            break
    out = {"workload": "realistic 128x128x64 -> 1024^2, 5x5 orders, spot S x S",
           "k_gather": k_gather, "k_fft": k_fft, "steps": steps,
           "l2": "flushed between timed runs (256 MiB write)",
           "rows": rows, "crossover_nnz_per_image": cross}
    with open(args.crossover, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({"crossover_nnz_per_image": cross,
                      "points": [(r["nnz_per_image"], round(r["gather_us_per_it"], 1),
                                  round(r["fft_us_per_it"], 1)) for r in rows]}), flush=True)


def main():
    args = parse_args()
    import synth
    if args.fma_peak:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(measure_fma_peak()), flush=True)
        return
    if args.crossover:
        run_crossover(args)
        return
    if args.paper_table:
        run_paper_table(args)
        return
    wl = synth.WORKLOADS[args.workload]
    k = args.k if args.k is not None else wl.k
    if args.impl == "reference":
        run_reference(args, wl, k)
    else:
        run_ours(args, wl, k)


if __name__ == "__main__":
    main()
