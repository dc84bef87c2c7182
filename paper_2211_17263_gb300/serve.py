"""Serving loop for concurrent inverse-rendering jobs (continuous batching).

Jobs arrive over time (each a workload: scene, target parameters, start parameters,
estimator settings, number of steps). The server keeps every admitted job resident on
the device -- scene, target image, parameters and Adam state -- and admits pending jobs
as soon as a slot and the context's HBM budget allow (a job that does not fit waits
until a finished job frees its memory). Each tick advances every active job by one
plateau-reduced gradient step:

  mode "batched": all active jobs' steps are packed into shared launches
                  (prdpt_step_batch: one sampler launch, one render launch per kind of job,
                  the path-sharing passes, one finalisation launch);
  mode "graphed": as "batched", but once the set of active jobs has stayed the same for
                  a tick, the packed step is captured as a CUDA graph and replayed (one
                  graph launch per tick) until the set changes;
  mode "plain":   one job per launch sequence (prdpt_step), jobs one after another.

Admission does not stall the device: the scene and the job's state are uploaded on the
library's own stream, and the target image is rendered at the job's reference
parameters straight into the job's device buffer on a side stream
(prdpt_job_render_target); the job's first step waits for that render by an event. The
host runs up to `ahead` ticks in front of the device and waits only for the oldest
tick's end event; a finished job is read and released once its last tick has completed
(reading waits for that job's work only, releasing does not wait).

Per-step latency is the device time from the start of the job's tick to the end of that
job's step (CUDA events). The report gives p50/p99 per-step latency, aggregate
job-steps/s, the peak number of co-resident jobs and the host time spent admitting.
Results do not depend on the mode or on the other jobs in the mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api, capi


@dataclass
class ServedJob:
    wl: object
    arrival: float
    steps: int
    scene: api.Scene | None = None
    job: api.Job | None = None
    ready: torch.cuda.Event | None = None  # the target render has completed
    done: int = 0
    latencies_ms: list = field(default_factory=list)
    admitted_at: float | None = None
    finished_at: float | None = None
    result: dict | None = None


def admit_job(ctx: api.Context, wl, side: torch.cuda.Stream, block_pixels: int = 0):
    """Upload the scene, create the resident job and enqueue its target render on `side`.
    Returns (scene, job, ready event) or None when the HBM budget refuses the job."""
    try:
        scene = ctx.upload_scene(wl.scene, wl.bindings)
    except capi.PrdptError as e:
        if e.code == capi.PRDPT_E_OUT_OF_BUDGET:
            return None
        raise
    try:
        job = api.Job(scene, wl, None, block_pixels=block_pixels)
    except capi.PrdptError as e:
        capi.prdpt_scene_release(ctx.handle, scene.id)
        if e.code == capi.PRDPT_E_OUT_OF_BUDGET:
            return None
        raise
    dev = torch.device("cuda", ctx.device)
    with torch.cuda.stream(side):
        host = torch.from_numpy(np.ascontiguousarray(wl.theta_ref, np.float32)).pin_memory()
        theta_ref = host.to(dev, non_blocking=True)
        job.render_target(theta_ref, stream=side)
        ready = torch.cuda.Event()
        ready.record(side)
    return scene, job, ready


def plain_capacity(ctx: api.Context, wls, steps_of, block_pixels: int = 0) -> dict:
    """The plain path's capacity on a mix, measured: one step of each job alone (after one
    warm-up step), timed with CUDA events; capacity = jobs / sum over jobs of steps x time."""
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    total_s = 0.0
    for wl in wls:
        got = admit_job(ctx, wl, side, block_pixels)
        if got is None:
            raise RuntimeError(f"job {wl.name} does not fit the HBM budget alone")
        scene, job, ready = got
        main.wait_event(ready)
        job.step(main)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        job.step(main)
        b.record(main)
        b.synchronize()
        total_s += steps_of(wl) * a.elapsed_time(b) * 1e-3
        job.release()
        capi.prdpt_scene_release(ctx.handle, scene.id)
    return {"jobs_per_s": len(wls) / total_s, "job_steps_per_s": sum(steps_of(w) for w in wls) / total_s,
            "method": "one timed step per job alone, x its steps"}


class Server:
    def __init__(self, ctx: api.Context, mode: str = "batched", max_active: int = 256, block_pixels: int = 0,
                 ahead: int = 2):
        if mode not in ("batched", "graphed", "plain"):
            raise ValueError("mode must be 'batched', 'graphed' or 'plain'")
        self.ctx = ctx
        self.mode = mode
        self.max_active = max_active
        self.block_pixels = block_pixels
        self.ahead = max(1, ahead)
        self.stream = torch.cuda.current_stream()
        self.side = torch.cuda.Stream()
        self._graph = None       # captured packed step of self._graph_ids
        self._graph_ids = None
        self._last_ids = None    # active set of the previous tick
        self.graph_replays = 0
        self.graph_captures = 0

    def _graphed_step(self, active):
        ids = tuple(sj.job.id for sj in active)
        if self._graph is not None and ids == self._graph_ids:
            self._graph.replay()
            self.graph_replays += 1
            return
        jobs = [sj.job for sj in active]
        api.step_batch(self.ctx, jobs, stream=self.stream)  # this tick's step (updates the descriptors)
        if ids == self._last_ids:  # stable set: capture the packed step for the next ticks
            self.stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                api.step_batch(self.ctx, jobs, stream=torch.cuda.current_stream())
            self._graph, self._graph_ids = g, ids
            self.graph_captures += 1
        else:
            self._graph, self._graph_ids = None, None
        self._last_ids = ids

    def _retire(self, sj: ServedJob, now: float):
        sj.result = sj.job.read()  # waits for this job's last step only
        sj.job.release()
        capi.prdpt_scene_release(self.ctx.handle, sj.scene.id)
        sj.job = None
        sj.finished_at = now

    def run(self, arrivals, steps_per_job=None, real_time: bool = True):
        """arrivals: list of (arrival_time_s, workload). Returns (report, jobs)."""
        jobs = [ServedJob(wl=wl, arrival=t, steps=int(steps_per_job(wl) if steps_per_job else wl.steps))
                for t, wl in sorted(arrivals, key=lambda a: a[0])]
        pending = collections.deque(jobs)
        active: list[ServedJob] = []
        inflight = collections.deque()  # (start event, [(job, end event)], jobs finishing at this tick)
        peak_active = 0
        peak_bytes = self.ctx.memory_used()
        ticks = 0
        admit_s = 0.0
        admitted = 0
        t0 = time.perf_counter()

        def complete_oldest():
            start, ends, finishing = inflight.popleft()
            ends[-1][1].synchronize()
            for sj, ev in ends:
                sj.latencies_ms.append(start.elapsed_time(ev))
            now = time.perf_counter() - t0
            for sj in finishing:
                self._retire(sj, now)

        while pending or active or inflight:
            now = time.perf_counter() - t0
            while pending and (not real_time or pending[0].arrival <= now) and len(active) < self.max_active:
                a0 = time.perf_counter()
                got = admit_job(self.ctx, pending[0].wl, self.side, self.block_pixels)
                admit_s += time.perf_counter() - a0
                if got is None:
                    break
                sj = pending.popleft()
                sj.scene, sj.job, sj.ready = got
                sj.admitted_at = time.perf_counter() - t0
                self.stream.wait_event(sj.ready)  # the first step after the target render
                active.append(sj)
                admitted += 1
            if not active:
                if inflight:
                    complete_oldest()  # frees memory for a job the budget refused
                    continue
                if pending and (not real_time or pending[0].arrival <= now):
                    raise RuntimeError(f"job {pending[0].wl.name} does not fit the HBM budget even alone")
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.01)))
                continue
            peak_active = max(peak_active, len(active))
            peak_bytes = max(peak_bytes, self.ctx.memory_used())
            start = torch.cuda.Event(enable_timing=True)
            start.record(self.stream)
            ends = []
            if self.mode in ("batched", "graphed"):
                if self.mode == "graphed":
                    self._graphed_step(active)
                else:
                    api.step_batch(self.ctx, [sj.job for sj in active], stream=self.stream)
                end = torch.cuda.Event(enable_timing=True)
                end.record(self.stream)
                ends = [(sj, end) for sj in active]
            else:
                for sj in active:
                    sj.job.step(self.stream)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(self.stream)
                    ends.append((sj, ev))
            ticks += 1
            finishing, still = [], []
            for sj in active:
                sj.done += 1
                (finishing if sj.done >= sj.steps else still).append(sj)
            active = still
            inflight.append((start, ends, finishing))
            while len(inflight) > self.ahead:
                complete_oldest()
        wall = time.perf_counter() - t0
        lat = np.concatenate([np.asarray(sj.latencies_ms) for sj in jobs]) if jobs else np.zeros(0)
        total_steps = int(sum(sj.done for sj in jobs))
        paths = float(sum(sj.done * sj.wl.paths_per_step for sj in jobs))
        report = {
            "mode": self.mode, "jobs": len(jobs), "job_steps": total_steps, "ticks": ticks, "wall_s": wall,
            "steps_per_s": total_steps / wall if wall > 0 else 0.0,
            "mpaths_per_s": paths / wall / 1e6 if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "peak_active": peak_active, "peak_hbm_bytes": peak_bytes,
            "graph_replays": self.graph_replays, "graph_captures": self.graph_captures,
            "admission_ms_mean": 1e3 * admit_s / max(admitted, 1), "admission_s_total": admit_s,
        }
        return report, jobs
