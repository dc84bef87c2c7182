"""Benchmark: plateau-reduced gradient steps on one GB300 (or N replicas under torchrun).

A step is one pass of the whole hot path on a resident job: draw the antithetic
perturbations (Sec. 3.2), bind theta +- tau into the scene, path-trace the R
perturbed renders with the per-pixel loss reduced inside the render kernel, form
the gradient of Eq. 10 and apply Adam -- all on the device.

Workload: the occlusion scene (256x256, three diffuse spheres and a 0.4^3 box on a
plane under a 1x1 area light, depth 4, 16 spp, theta = box centre, sigma = 0.05,
N = 16 renders = 8 antithetic pairs), synthetic and seeded.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "smoothed-gradient steps/s"
UNIT = "steps/s"
# Algorithmic FP32 operations (add/sub/mul = 1, fma = 2, div/sqrt/rsqrt = 1; compares
# and min/max not counted) per unit of work of the path tracer.
FLOPS = {"sphere_test": 22, "quad_test": 32, "box_test": 12, "path": 27, "vertex": 120}
WORKLOADS = {"small": "config_small", "occlusion": "config_occlusion", "gi_box": "config_gi_box",
             "caustic": "config_caustic",
             # the pathwise estimator (Eq. 9) on material parameters
             "small_albedo": "config_small_albedo", "gi_albedo": "config_gi_albedo",
             # the 128 x 128 RGB texture: 49,152 parameters
             "texture": "config_texture"}


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
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
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _code_only(text):
    """Source text without // comments and blank lines (comment edits do not change a kernel)."""
    lines = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip() if "//" in line and '"' not in line.split("//", 1)[0] else line.rstrip()
        if code.strip():
            lines.append(code)
    return "\n".join(lines)


def _kernel_source_sha(read=None):
    """Hash of the kernel sources' code; a profile summary is used only while it matches."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "internal.h"):
        path = os.path.join("paper_2211_17263_gb300", "csrc", f)
        text = read(path) if read else open(os.path.join(ROOT, path)).read()
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


def _profiled(workload_name, key):
    """A per-step figure of the occlusion workload's render kernels from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    if not workload_name.startswith("occlusion"):
        return None
    path = os.path.join(ROOT, "profiles", "render_pipeline_occlusion-256x256_ncu.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().split("`")[1] if "`" in v else v.strip()
    if vals.get("kernel_source_sha") != _kernel_source_sha():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


CPU_SAMPLE_MAX_PATHS = 40_000_000  # larger steps are sampled (one pair, 4 spp) and scaled


def _issue_rate(workload_name, sms, sm_mhz, pipeline_ms, per_render_ms):
    peak = 4.0 * sms * sm_mhz * 1e6 / 1e9  # G warp instructions / s
    out = {"unit": "G warp instr/s", "peak": peak}
    for key, ms, name in (("warp_instructions_per_step", pipeline_ms, "pipeline"),
                          ("warp_instructions_per_step_no_sharing", per_render_ms, "per_render_kernel")):
        n = _profiled(workload_name, key)
        if n is None or not ms:
            return None
        out[name] = n / (ms * 1e-3) / 1e9
        out[name + "_frac"] = out[name] / peak
    return out


def cpu_baseline(wl, target, nthreads=0, budget_s=10.0, max_steps=20):
    """The FP64 oracle on whole steps of the same workload, repeated until about
    `budget_s` seconds of wall time have passed (bounded by `max_steps`). A step of
    more than CPU_SAMPLE_MAX_PATHS paths is sampled instead: one antithetic pair at
    4 spp, its time scaled by the ratio of path counts."""
    import oracle
    import workloads
    cores = nthreads or os.cpu_count() or 1
    run, scale, what = wl, 1.0, "whole steps"
    if wl.paths_per_step > CPU_SAMPLE_MAX_PATHS:
        run = workloads.scaled(wl, spp=4, pairs=1)
        scale = wl.paths_per_step / run.paths_per_step
        what = f"sampled steps (1 pair, 4 spp; time x{scale:.0f} by path count)"
    estimate = oracle.kdp_grad if getattr(wl, "estimator", 0) == 1 else oracle.smoothed_grad
    n, t0 = 0, time.perf_counter()
    while n < max_steps and (n == 0 or time.perf_counter() - t0 < budget_s):
        estimate(run, target=target, nthreads=cores, step=n)
        n += 1
    dt = (time.perf_counter() - t0) / n * scale
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} {what} ({wl.renders} renders at {wl.width}x{wl.height}, {wl.spp} spp), "
                      f"{dt:.2f} s per full step", "cpu_model": _cpu_model()}


def serving_bench(device, n_jobs, steps_per_job, gpaths_per_s, seed=0):
    """Serving mix (jobs drawn from the small, occlusion and GI-box workloads with random
    resolution 128-512, N in {8,16,32,64} renders, spp in {8,...,64}): Poisson arrivals at
    1.5x the plain path's estimated capacity, served one job per launch ("plain") and with
    continuous batching ("batched"), on the same arrival sequence."""
    import workloads
    from paper_2211_17263_gb300 import api
    from paper_2211_17263_gb300.serve import Server

    base = workloads.serving_mix(n_jobs=n_jobs, seed=seed)
    mean_paths = float(np.mean([wl.paths_per_step for _, wl in base])) * steps_per_job
    capacity_jobs_per_s = gpaths_per_s * 1e9 / mean_paths
    rate = 1.5 * capacity_jobs_per_s
    rng = np.random.default_rng(seed + 7)
    t, arrivals = 0.0, []
    for _, wl in base:
        t += float(rng.exponential(1.0 / rate))
        arrivals.append((t, wl))
    out = {"jobs": n_jobs, "steps_per_job": steps_per_job, "arrival_rate_jobs_per_s": rate,
           "hbm_budget_bytes": 150 * 10 ** 9}
    for mode in ("plain", "batched", "graphed"):
        ctx = api.Context(device, hbm_budget_bytes=150 * 10 ** 9)
        try:
            rep, _ = Server(ctx, mode=mode, max_active=256).run(arrivals, steps_per_job=lambda wl: steps_per_job)
        finally:
            ctx.close()
        out[mode] = {k: rep[k] for k in ("steps_per_s", "mpaths_per_s", "p50_ms", "p99_ms", "peak_active", "wall_s",
                                         "graph_replays")}
    out["batched_over_plain"] = out["batched"]["steps_per_s"] / out["plain"]["steps_per_s"]
    out["graphed_over_plain"] = out["graphed"]["steps_per_s"] / out["plain"]["steps_per_s"]
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, timed as it stands on the host cores."""
    if rank != 0:
        return
    import oracle
    import workloads
    wl = workloads.config_occlusion()
    target = oracle.render_target(wl)
    cores = os.cpu_count() or 1
    # whole steps while K of them fit in about 100 s; else each step is a bounded sample
    # (one pair at 4 spp) whose time is scaled by the ratio of path counts
    t0 = time.perf_counter()
    oracle.smoothed_grad(wl, target=target, nthreads=cores, step=0)
    full = time.perf_counter() - t0
    run, scale, what = wl, 1.0, "whole steps"
    if full * args.steps > 100.0:
        run = workloads.scaled(wl, spp=4, pairs=1)
        scale = wl.paths_per_step / run.paths_per_step
        what = f"sampled steps (1 pair, 4 spp; time x{scale:.0f} by path count)"
    for _ in range(args.warmup):
        oracle.smoothed_grad(run, target=target, nthreads=cores, step=0)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.smoothed_grad(run, target=target, nthreads=cores, step=k)
    dt = (time.perf_counter() - t0) / args.steps * scale
    value = 1.0 / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "renders": wl.renders, "pairs": wl.pairs, "width": wl.width,
                   "height": wl.height, "spp": wl.spp, "depth": wl.depth, "D": wl.D, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} {what} ({wl.renders} renders at {wl.width}x{wl.height}, "
                                   f"{wl.spp} spp)", "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--block-pixels", type=int, default=0, help="pixels per warp work item (8, 16, 32; 0 = auto)")
    ap.add_argument("--serving-jobs", type=int, default=64, help="jobs in the serving mix (0 = skip serving)")
    ap.add_argument("--serving-steps", type=int, default=4, help="steps per served job")
    ap.add_argument("--workload", default="occlusion", choices=sorted(WORKLOADS),
                    help="occlusion is the headline workload; the others are measured on request")
    ap.add_argument("--estimator", default="auto", choices=["auto", "kernel", "pathwise"],
                    help="auto: the workload's own; kernel: Eq. 10 with the radial sampler; pathwise: Eq. 9 "
                         "(Gaussian draws; material bindings only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2211_17263_gb300 import dist as pdist
    rank, world, local = pdist.env_rank()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    import workloads
    from paper_2211_17263_gb300 import api

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        pdist.barrier(world)

    wl = getattr(workloads, WORKLOADS[args.workload])(seed=rank)  # one independent replica per rank
    if args.estimator == "kernel":
        wl.estimator, wl.sampler = 0, workloads.SAMPLER_RADIAL
    elif args.estimator == "pathwise":
        wl.estimator, wl.sampler = 1, workloads.SAMPLER_GAUSS
    ctx = api.Context(local)
    probe_tflops, probe_ms = ctx.fp32_peak_probe()  # FMA-chain launch: confirms the FP32 peak
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=f"cuda:{local}")  # noqa: E731
    target = scene.render_batch(dev(wl.theta_ref[None]), wl.width, wl.height, wl.spp, wl.depth, wl.rr_start,
                                seed=wl.seed, step=0, tag=3, crn=1)[0]
    target_host = target.cpu().numpy()
    job = api.Job(scene, wl, target_host, block_pixels=args.block_pixels)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        job.step(stream)
    torch.cuda.synchronize()

    # algorithmic work of one step (counting kernel variant, untimed)
    ctx.counters_enable(True)
    job.step(stream)
    counts = ctx.counters_read()
    ctx.counters_enable(False)
    flops_step = (counts[0] * FLOPS["sphere_test"] + counts[1] * FLOPS["quad_test"] + counts[2] * FLOPS["box_test"]
                  + counts[3] * FLOPS["path"] + counts[4] * FLOPS["vertex"])

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{local}")  # 256 MB > L2
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ctx.kernel_timing(True)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the timed events)
        starts[k].record(stream)
        job.step(stream)
        ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    trace_ms, launches = ctx.kernel_timing_read()
    ctx.kernel_timing(False)
    step_ms = pdist.max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps, world,
                                   device=f"cuda:{local}")
    state = job.read()

    # the per-render kernel on the same workload (path sharing off): its own roofline
    plain_job = api.Job(scene, wl, target_host, block_pixels=args.block_pixels, no_path_sharing=1)
    for _ in range(3):
        plain_job.step(stream)
    ctx.counters_enable(True)
    plain_job.step(stream)
    pcounts = ctx.counters_read()
    ctx.counters_enable(False)
    torch.cuda.synchronize()
    ctx.kernel_timing(True)
    n_plain = min(args.steps, 100)
    for _ in range(n_plain):
        flush.zero_()
        plain_job.step(stream)
    p_ms, p_launches = ctx.kernel_timing_read()
    ctx.kernel_timing(False)
    plain_job.release()
    pflops = (pcounts[0] * FLOPS["sphere_test"] + pcounts[1] * FLOPS["quad_test"] + pcounts[2] * FLOPS["box_test"]
              + pcounts[3] * FLOPS["path"] + pcounts[4] * FLOPS["vertex"])

    # end to end through the C ABI with host buffers: H2D inputs, gradient, Adam, D2H results
    e2e = None
    # through the C ABI with host buffers (prdpt_step_host): each step uploads theta, Adam's
    # m and v, sigma and the target from page-locked memory, computes the gradient, applies
    # Adam on the device and downloads theta, m, v, the gradient and the losses
    D, R, npx4 = wl.D, wl.renders, 4 * wl.width * wl.height
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()  # noqa: E731
    theta_h, sigma_h, target_h = pin(wl.theta0), pin(wl.sigma), pin(target_host)
    m_h, v_h, g_h, L_h = pin(np.zeros(D)), pin(np.zeros(D)), pin(np.zeros(D)), pin(np.zeros(R))
    h2d = 4 * (npx4 + 4 * D + 1)  # target; sigma, Adam's step, theta, m, v in one staged copy
    d2h = 4 * (4 * D + R)  # theta, m, v, gradient, losses in one copy
    opts = scene.grad_opts(wl, step=0)

    def e2e_step(k):
        opts.step = k
        scene.step_host(theta_h, m_h, v_h, k + 1, wl.lr, sigma_h, target_h, opts, grad=g_h, losses=L_h)

    for k in range(args.warmup):
        e2e_step(k)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    e2e_s = pdist.max_over_ranks((time.perf_counter() - t0) / args.steps, world, device=f"cuda:{local}")
    e2e = {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    if rank == 0:
        peaks = _measured_peaks()
        props = torch.cuda.get_device_properties(local)
        sm_max = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
        fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
        trace_avg_ms = trace_ms / max(launches, 1)
        achieved = flops_step / (trace_avg_ms * 1e-3) / 1e12
        p_avg_ms = p_ms / max(p_launches, 1)
        p_achieved = pflops / (p_avg_ms * 1e-3) / 1e12
        value = world * 1000.0 / step_ms
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "renders": wl.renders, "pairs": wl.pairs, "width": wl.width,
                       "height": wl.height, "spp": wl.spp, "depth": wl.depth, "D": wl.D,
                       "estimator": "Eq. 9 (pathwise)" if getattr(wl, "estimator", 0) == 1 else "Eq. 10",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
            "mpaths_per_s": world * wl.paths_per_step / (step_ms * 1e-3) / 1e6,
            # ray segments (closest-hit rays + shadow rays) traced per second: as executed
            # (shared pass + re-traced paths) and as the method defines them (every render)
            "msegments_per_s": world * (counts[5] + counts[6]) / (step_ms * 1e-3) / 1e6,
            "msegments_per_s_method": world * (pcounts[5] + pcounts[6]) / (step_ms * 1e-3) / 1e6,
            "wall_s": wall,
            "render_kernel_ms": trace_avg_ms,
            "work_per_step": {"sphere_tests": counts[0], "quad_tests": counts[1], "box_tests": counts[2],
                              "paths": counts[3], "vertices": counts[4], "shadow_rays": counts[5],
                              "closest_hit_rays": counts[6]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": _profiled(wl.name, "dram_bytes_per_step"),
                         "kernel": ("render pipeline (k_trace shared pass, k_trace_affected, k_shared_epilogue,"
                                    " k_finalize)" if counts[3] < wl.paths_per_step else "k_trace + k_finalize"),
                         "peak_basis": f"FP32 FMA: {props.multi_processor_count} SMs x 128 lanes"
                                       f" x 2 flop x {sm_max:.0f} MHz"},
            "roofline_per_render_kernel": {
                "bound": "alu", "achieved": p_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": p_achieved / fp32_peak, "kernel": "k_trace (path sharing off) + k_finalize",
                "ms_per_step": p_avg_ms, "paths_per_step": pcounts[3]},
            # diagnostic beside the algorithmic roofline: warp instructions issued per second
            # (ncu count per step from the committed summary) against 4 schedulers x SMs x clock
            "issue_rate": _issue_rate(wl.name, props.multi_processor_count, sm_max, trace_avg_ms, p_avg_ms),
            "fp32_probe": {"achieved_tflops": probe_tflops, "ms": probe_ms,
                           "frac_of_peak": probe_tflops / fp32_peak},
            "e2e": e2e,
            # sampler, render kernel(s), finalisation; path sharing adds the per-render and
            # epilogue passes; texture scenes add the D-dimensional draws and gradient kernels
            "gpu_launches": ((5 if counts[3] < wl.paths_per_step else 3)
                             + ((3 if wl.sampler == workloads.SAMPLER_RADIAL else 2) if wl.D > 64 else 0)) * args.steps,
            "clocks": clocks,
            "final_loss_mean": float(np.mean(state["losses"])),
        }
        if world == 1 and args.serving_jobs > 0 and args.workload == "occlusion":
            line["serving"] = serving_bench(local, args.serving_jobs, args.serving_steps,
                                            line["mpaths_per_s"] / 1000.0)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, target_host)
            # the same oracle on one thread (one bounded sample), beside the all-core figure
            one = cpu_baseline(wl, target_host, nthreads=1, budget_s=3.0, max_steps=1)
            line["cpu_baseline"]["single_thread"] = {"value": one["value"], "unit": one["unit"],
                                                     "sample": one["sample"]}
        print(json.dumps(line), flush=True)
    job.release()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
