"""Benchmark: plateau-reduced gradient steps on one GB300 (or N replicas under torchrun).

A step is one pass of the whole hot path on a resident job: draw the antithetic
perturbations (Sec. 3.2), bind theta +- tau into the scene, path-trace the R
perturbed renders with the per-pixel loss reduced inside the render kernel, form
the gradient of Eq. 10 and apply Adam -- all on the device.

Workload (default): the caustic task, the largest single-GPU configuration -- a
512x512 image of a glass sphere (IOR 1.5) above a diffuse floor lit by a small
0.2x0.2 area light, path depth 12 with Russian roulette from the 4th vertex,
theta = light position (3-D), sigma = 0.125, N = 64 renders (32 antithetic pairs) x
64 spp = 1.07 G paths per step; synthetic and seeded. `--workload` measures the
other workloads (occlusion 256^2, GI box 512^2, small 64^2, texture, Eq. 9 ones).
The serving mix (continuous batching of concurrent jobs) is measured beside it.

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


def _profile_path(workload_name):
    return os.path.join(ROOT, "profiles", f"render_pipeline_{workload_name}_ncu.md")


def _profiled(workload_name, key):
    """A per-step figure of the workload's render kernels from the committed ncu summary
    profiles/render_pipeline_<workload>_ncu.md, if it was taken on the current kernel
    source (hash of the code without comments); else None."""
    try:
        text = open(_profile_path(workload_name)).read()
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


def _emitter_bound(wl):
    """Does a position or radius binding move an emitter (the emitter-sharing mode's jobs;
    geometry-only jobs share paths through the shared-pass pipeline)?"""
    import workloads
    sc = wl.scene
    for kind, idx, _ in np.asarray(wl.bindings):
        if kind in (workloads.BIND_PRIM_POS, workloads.BIND_SPHERE_RADIUS):
            if np.any(sc.mat_param[sc.prim_mat[idx], 3:6] > 0):
                return True
    return False


def _launches_per_step(wl, sharing):
    """The library's kernel launches in one resident step: sampler, render kernel,
    finalisation; path sharing adds the per-render and epilogue passes (emitter sharing runs
    one render kernel); texture scenes add the D-dimensional draws and gradient kernels."""
    import workloads
    n = 5 if sharing and not _emitter_bound(wl) else 3
    if wl.D > 64:
        n += 3 if wl.sampler == workloads.SAMPLER_RADIAL else 2
    return n


CPU_SAMPLE_MAX_PATHS = 40_000_000  # larger steps are sampled (one pair, 4 spp) and scaled


def _issue_rate(workload_name, sms, sm_mhz, pipeline_ms, per_render_ms):
    """Warp instructions issued per second against 4 schedulers x SMs x clock: counts per
    step from the committed ncu summary (None unless its kernel source hash matches),
    times from this run."""
    peak = 4.0 * sms * sm_mhz * 1e6 / 1e9  # G warp instructions / s
    out = {"unit": "G warp instr/s", "peak": peak}
    for key, ms, name in (("warp_instructions_per_step", pipeline_ms, "pipeline"),
                          ("warp_instructions_per_step_no_sharing", per_render_ms, "per_render_kernel")):
        n = _profiled(workload_name, key)
        if n is None or not ms:
            if name == "pipeline":
                return None
            continue
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


def serving_bench(device, n_jobs, steps_per_job, modes, seed=0):
    """Serving mix (jobs drawn from the small, occlusion and GI-box workloads with random
    resolution 128-512, N in {8,16,32,64} renders, spp in {8,...,64}; 100 steps per job, 300
    for GI-box jobs, unless steps_per_job is given): Poisson arrivals at 1.5x the plain
    path's capacity, measured first from one timed step of each job alone, served one job
    per launch ("plain"), packed ("batched") and packed with CUDA-graph replay ("graphed"),
    on the same arrival sequence."""
    import workloads
    from paper_2211_17263_gb300 import api
    from paper_2211_17263_gb300.serve import Server, plain_capacity

    base = workloads.serving_mix(n_jobs=n_jobs, seed=seed)
    steps_of = (lambda wl: steps_per_job) if steps_per_job else (lambda wl: wl.steps)
    ctx = api.Context(device, hbm_budget_bytes=150 * 10 ** 9)
    try:
        cap = plain_capacity(ctx, [wl for _, wl in base], steps_of)
    finally:
        ctx.close()
    rate = 1.5 * cap["jobs_per_s"]
    rng = np.random.default_rng(seed + 7)
    t, arrivals = 0.0, []
    for _, wl in base:
        t += float(rng.exponential(1.0 / rate))
        arrivals.append((t, wl))
    out = {"jobs": n_jobs, "job_steps": int(sum(steps_of(wl) for _, wl in base)),
           "steps_per_job": steps_per_job or "100 (GI box: 300)",
           "subset": "the first n jobs of the 256-job mix" if n_jobs < 256 else "the full mix",
           "plain_capacity": cap, "arrival_rate_jobs_per_s": rate, "hbm_budget_bytes": 150 * 10 ** 9}
    for mode in modes:
        ctx = api.Context(device, hbm_budget_bytes=150 * 10 ** 9)
        try:
            rep, _ = Server(ctx, mode=mode, max_active=256).run(arrivals, steps_per_job=steps_of)
        finally:
            ctx.close()
        out[mode] = {k: rep[k] for k in ("steps_per_s", "mpaths_per_s", "p50_ms", "p99_ms", "peak_active", "wall_s",
                                         "graph_replays", "graph_captures", "admission_ms_mean", "ticks")
                     if k in rep}
    if "plain" in out:
        for mode in modes:
            if mode != "plain":
                out[f"{mode}_over_plain"] = out[mode]["steps_per_s"] / out["plain"]["steps_per_s"]
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, timed as it stands on the host cores."""
    if rank != 0:
        return
    import oracle
    import workloads
    wl = getattr(workloads, WORKLOADS[args.workload])()
    cores = os.cpu_count() or 1
    target = oracle.render_target(wl, nthreads=cores)
    # whole steps while K of them fit in about 100 s; else (and always above
    # CPU_SAMPLE_MAX_PATHS paths per step) each step is a bounded sample -- one pair at
    # 4 spp -- whose time is scaled by the ratio of path counts
    run, scale, what = wl, 1.0, "whole steps"
    full = float("inf")
    if wl.paths_per_step <= CPU_SAMPLE_MAX_PATHS:
        t0 = time.perf_counter()
        oracle.smoothed_grad(wl, target=target, nthreads=cores, step=0)
        full = time.perf_counter() - t0
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
    ap.add_argument("--reduce", default="",
                    help="W,H,SPP,PAIRS: run a reduced case of the workload (profiling only; the line says so)")
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--block-pixels", type=int, default=0,
                    help="pixels per warp work item (8, 16, 32; 0 = the autotuned or default shape)")
    ap.add_argument("--render-groups", type=int, default=0,
                    help="with --block-pixels: renders traced side by side per warp (0 = automatic, -1 = off)")
    ap.add_argument("--serving-jobs", type=int, default=12,
                    help="jobs of the serving mix served in each mode (0 = skip serving); 256 is the full mix")
    ap.add_argument("--serving-steps", type=int, default=0,
                    help="steps per served job (0 = the mix's own: 100, and 300 for GI-box jobs)")
    ap.add_argument("--serving-modes", default="plain,batched,graphed")
    ap.add_argument("--workload", default="caustic", choices=sorted(WORKLOADS),
                    help="caustic (512^2, 64 renders x 64 spp, depth 12) is the headline; the others on request")
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
    from paper_2211_17263_gb300 import api, autotune

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        pdist.barrier(world)

    wl = getattr(workloads, WORKLOADS[args.workload])(seed=rank)  # one independent replica per rank
    if args.reduce:  # a reduced case of the workload, for profiling (not a bench line)
        w, h, spp, pairs = (int(x) for x in args.reduce.split(","))
        wl = workloads.scaled(wl, width=w, height=h, spp=spp, pairs=pairs)
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
    # launch shape: given, else the autotuner's choice for this workload shape (tuned now if
    # the cache has no entry; the tuning steps run before and outside the timed region)
    tuned = None
    if args.block_pixels:
        shape = {"block_pixels": args.block_pixels, "ctas_per_sm": 0, "render_groups": args.render_groups,
                 "no_path_sharing": 0, "source": "--block-pixels"}
    else:
        tuned = autotune.autotune(scene, wl, target_host)
        shape = {"block_pixels": tuned["block_pixels"], "ctas_per_sm": tuned["ctas_per_sm"],
                 "render_groups": tuned.get("render_groups", 0), "no_path_sharing": tuned.get("no_path_sharing", 0),
                 "source": "autotuner (cached)" if tuned["cached"] else "autotuner"}
    job = api.Job(scene, wl, target_host, block_pixels=shape["block_pixels"], ctas_per_sm=shape["ctas_per_sm"],
                  render_groups=shape["render_groups"], no_path_sharing=shape["no_path_sharing"], use_tuned=False)
    stream = torch.cuda.current_stream()
    # warm-up: at least W steps and at least one second of device work (clocks ramp up
    # under sustained load; a few short steps after start-up run slow), each after an L2
    # flush as the timed steps are (so a profiler sees warm-up steps as timed ones)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{local}")  # 256 MB > L2
    t_warm, n_warm = time.perf_counter(), 0
    while n_warm < args.warmup or time.perf_counter() - t_warm < 1.0:
        flush.zero_()
        job.step(stream)
        n_warm += 1
        if n_warm % 4 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()

    # algorithmic work of one step (counting kernel variant, untimed)
    ctx.counters_enable(True)
    job.step(stream)
    counts = ctx.counters_read()
    ctx.counters_enable(False)
    flops_step = (counts[0] * FLOPS["sphere_test"] + counts[1] * FLOPS["quad_test"] + counts[2] * FLOPS["box_test"]
                  + counts[3] * FLOPS["path"] + counts[4] * FLOPS["vertex"])
    sharing = counts[3] < wl.paths_per_step  # path sharing traces fewer paths than R x H x W x S

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    # the device idled while the sampler started: a short re-warm so that the first timed
    # steps do not run at a lowered clock
    t_rw, n_rw = time.perf_counter(), 0
    while time.perf_counter() - t_rw < 0.2:
        flush.zero_()
        job.step(stream)
        n_rw += 1
        torch.cuda.synchronize()
    n_before = n_warm + 1 + n_rw  # steps the job took before its timed ones
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
    per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    step_ms = pdist.max_over_ranks(sum(per_step) / args.steps, world, device=f"cuda:{local}")
    state = job.read()

    # with path sharing: the per-render kernel on the same workload (sharing off), its own
    # roofline; without, the timed step already is the per-render kernel
    per_render = None
    if sharing:
        plain_job = api.Job(scene, wl, target_host, block_pixels=shape["block_pixels"],
                            ctas_per_sm=shape["ctas_per_sm"], no_path_sharing=1, render_groups=-1, use_tuned=False)
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
        pflops = (pcounts[0] * FLOPS["sphere_test"] + pcounts[1] * FLOPS["quad_test"]
                  + pcounts[2] * FLOPS["box_test"] + pcounts[3] * FLOPS["path"] + pcounts[4] * FLOPS["vertex"])
        per_render = {"counts": pcounts, "ms": p_ms / max(p_launches, 1), "flops": pflops}

    # end to end through the C ABI with host buffers (prdpt_step_host): each step uploads
    # theta, Adam's m and v, sigma and the target from page-locked memory, computes the
    # gradient, applies Adam on the device and downloads theta, m, v, the gradient and the losses.
    # The cost of a step depends on theta (the caustic step takes 7.6 ms at theta0 and 6.7 ms
    # some 200 steps on), so the leg first takes, untimed, as many steps from theta0 as the
    # resident job took before its timed steps: both then time the same stretch of the descent
    D, R, npx4 = wl.D, wl.renders, 4 * wl.width * wl.height
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()  # noqa: E731
    theta_h, sigma_h, target_h = pin(wl.theta0), pin(wl.sigma), pin(target_host)
    m_h, v_h, g_h, L_h = pin(np.zeros(D)), pin(np.zeros(D)), pin(np.zeros(D)), pin(np.zeros(R))
    h2d = 4 * (npx4 + 4 * D + 1)  # target; sigma, Adam's step, theta, m, v in one staged copy
    d2h = 4 * (4 * D + R)  # theta, m, v, gradient, losses in one copy
    opts = scene.grad_opts(wl, step=0, block_pixels=shape["block_pixels"], ctas_per_sm=shape["ctas_per_sm"],
                           render_groups=shape["render_groups"], no_path_sharing=shape["no_path_sharing"])

    def e2e_step(k):
        opts.step = k
        scene.step_host(theta_h, m_h, v_h, k + 1, wl.lr, sigma_h, target_h, opts, grad=g_h, losses=L_h)

    for k in range(max(args.warmup, n_before)):
        e2e_step(k)
    barrier()
    torch.cuda.synchronize()
    k0 = max(args.warmup, n_before)
    t0 = time.perf_counter()
    for k in range(k0, k0 + args.steps):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    e2e_s = pdist.max_over_ranks((time.perf_counter() - t0) / args.steps, world, device=f"cuda:{local}")
    e2e = {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "call": "prdpt_step_host", "steps_before_timed": k0}

    if rank == 0:
        peaks = _measured_peaks()
        props = torch.cuda.get_device_properties(local)
        sm_max = float(peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0)
        fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
        trace_avg_ms = trace_ms / max(launches, 1)
        model_achieved = flops_step / (trace_avg_ms * 1e-3) / 1e12
        # FP32 flop per step counted by ncu (2 x FFMA + FADD + FMUL thread instructions of the
        # step's render kernel) when the committed summary was taken on these kernel sources;
        # else the work-counter model
        fp32_counted = _profiled(wl.name, "fp32_flop_per_step")
        achieved = fp32_counted / (trace_avg_ms * 1e-3) / 1e12 if fp32_counted else model_achieved
        value = world * 1000.0 / step_ms
        traffic = _profiled(wl.name, "dram_bytes_per_step")
        if sharing and _emitter_bound(wl):
            kernels = "emitter-sharing kernel k_trace_emit + k_finalize"
        elif sharing:
            kernels = "render pipeline (k_trace shared pass, k_trace_affected, k_shared_epilogue, k_finalize)"
        elif shape["render_groups"] >= 0 and wl.crn and wl.D <= 64:
            kernels = "render-group kernel k_trace_group + k_finalize"
        else:
            kernels = "render kernel k_trace + k_finalize"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "renders": wl.renders, "pairs": wl.pairs, "width": wl.width,
                       "height": wl.height, "spp": wl.spp, "depth": wl.depth, "rr_start": wl.rr_start, "D": wl.D,
                       "estimator": "Eq. 9 (pathwise)" if getattr(wl, "estimator", 0) == 1 else "Eq. 10",
                       "launch_shape": shape, "path_sharing": bool(sharing),
                       "reduced": bool(args.reduce),
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
            # paths of the method per second: R x H x W x S per step; with path sharing
            # ("effective") fewer are traced -- mpaths_traced_per_s counts those
            "mpaths_per_s": world * wl.paths_per_step / (step_ms * 1e-3) / 1e6,
            "mpaths_per_s_kind": "effective (R x H x W x S per step; path sharing traces fewer)" if sharing
                                 else "traced (R x H x W x S per step, every path traced)",
            "mpaths_traced_per_s": world * counts[3] / (step_ms * 1e-3) / 1e6,
            # ray segments (closest-hit rays + shadow rays) traced per second
            "msegments_per_s": world * (counts[5] + counts[6]) / (step_ms * 1e-3) / 1e6,
            "wall_s": wall,
            "step_ms_min_median_max": [float(np.min(per_step)), float(np.median(per_step)), float(np.max(per_step))],
            "warmup_steps_run": n_warm,
            "render_kernel_ms": trace_avg_ms,
            "work_per_step": {"sphere_tests": counts[0], "quad_tests": counts[1], "box_tests": counts[2],
                              "paths": counts[3], "vertices": counts[4], "shadow_rays": counts[5],
                              "closest_hit_rays": counts[6]},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": traffic,
                         "traffic_source": (f"ncu, profiles/{os.path.basename(_profile_path(wl.name))} (kernel "
                                            "source hash matches)") if traffic is not None else None,
                         "kernel": kernels,
                         "achieved_basis": ("ncu-counted FP32 flop per step (2 FFMA + FADD + FMUL, profiles/, "
                                            "kernel source hash matches) / mean CUDA-event time of the step's "
                                            "kernels") if fp32_counted else
                                           ("model FP32 flop per step from the kernels' work counters / mean "
                                            "CUDA-event time of the step's kernels"),
                         "model_achieved": model_achieved,
                         "peak_basis": f"FP32 FMA: {props.multi_processor_count} SMs x 128 lanes"
                                       f" x 2 flop x {sm_max:.0f} MHz"},
            "fp32_probe": {"achieved_tflops": probe_tflops, "ms": probe_ms,
                           "frac_of_peak": probe_tflops / fp32_peak},
            "e2e": e2e,
            "gpu_launches": _launches_per_step(wl, sharing) * args.steps,
            "clocks": clocks,
            "final_loss_mean": float(np.mean(state["losses"])),
        }
        if per_render is not None:
            p_achieved = per_render["flops"] / (per_render["ms"] * 1e-3) / 1e12
            line["roofline_per_render_kernel"] = {
                "bound": "alu", "achieved": p_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": p_achieved / fp32_peak, "kernel": "k_trace (path sharing off) + k_finalize",
                "ms_per_step": per_render["ms"], "paths_per_step": per_render["counts"][3]}
            # the method's work (every render's paths traced, counted by the per-render kernel)
            # over this step's kernel time: what sharing buys, not a hardware efficiency
            e_achieved = per_render["flops"] / (trace_avg_ms * 1e-3) / 1e12
            line["roofline_effective"] = {
                "bound": "alu", "achieved": e_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": e_achieved / fp32_peak,
                "basis": "model FP32 flop of tracing every render's paths (the per-render kernel's work counters) "
                         "/ mean CUDA-event time of this step's kernels"}
        issue = _issue_rate(wl.name, props.multi_processor_count, sm_max, trace_avg_ms,
                            per_render["ms"] if per_render else None)
        if issue is not None:
            issue["source"] = "warp instructions per step from the committed ncu summary; times from this run"
        line["issue_rate"] = issue
        if tuned is not None:
            line["autotune"] = {"choice": {k: tuned.get(k) for k in ("block_pixels", "ctas_per_sm", "render_groups",
                                                                     "no_path_sharing")},
                                "cached": tuned["cached"], "ms": tuned.get("ms"),
                                "tried": tuned.get("tried")}
        if world == 1 and args.serving_jobs > 0:
            line["serving"] = serving_bench(local, args.serving_jobs, args.serving_steps,
                                            [m for m in args.serving_modes.split(",") if m])
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
