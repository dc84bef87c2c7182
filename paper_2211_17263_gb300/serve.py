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

Per-step latency is measured with CUDA events from the start of the tick (when the
step becomes runnable) to the completion of that job's step. The report gives p50/p99
per-step latency, aggregate job-steps/s and the peak number of co-resident jobs.
Results do not depend on the mode or on the other jobs in the mix.
"""
from __future__ import annotations

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
    done: int = 0
    latencies_ms: list = field(default_factory=list)
    admitted_at: float | None = None
    finished_at: float | None = None
    result: dict | None = None


class Server:
    def __init__(self, ctx: api.Context, mode: str = "batched", max_active: int = 256, block_pixels: int = 0):
        if mode not in ("batched", "graphed", "plain"):
            raise ValueError("mode must be 'batched', 'graphed' or 'plain'")
        self.ctx = ctx
        self.mode = mode
        self.max_active = max_active
        self.block_pixels = block_pixels
        self.stream = torch.cuda.current_stream()
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

    def _admit(self, sj: ServedJob) -> bool:
        wl = sj.wl
        try:
            scene = self.ctx.upload_scene(wl.scene, wl.bindings)
        except capi.PrdptError as e:
            if e.code == capi.PRDPT_E_OUT_OF_BUDGET:
                return False
            raise
        dev = torch.device("cuda", self.ctx.device)
        theta_ref = torch.as_tensor(np.ascontiguousarray(wl.theta_ref[None], np.float32), device=dev)
        target = scene.render_batch(theta_ref, wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, seed=wl.seed,
                                    step=0, tag=3, crn=1)[0].cpu().numpy()
        try:
            job = api.Job(scene, wl, target, block_pixels=self.block_pixels)
        except capi.PrdptError as e:
            capi.prdpt_scene_release(self.ctx.handle, scene.id)
            if e.code == capi.PRDPT_E_OUT_OF_BUDGET:
                return False
            raise
        sj.scene, sj.job = scene, job
        return True

    def _retire(self, sj: ServedJob, now: float):
        sj.result = sj.job.read()
        sj.job.release()
        capi.prdpt_scene_release(self.ctx.handle, sj.scene.id)
        sj.job = None
        sj.finished_at = now

    def run(self, arrivals, steps_per_job=None, real_time: bool = True) -> dict:
        """arrivals: list of (arrival_time_s, workload). Returns the report and the jobs."""
        jobs = [ServedJob(wl=wl, arrival=t, steps=int(steps_per_job(wl) if steps_per_job else wl.steps))
                for t, wl in sorted(arrivals, key=lambda a: a[0])]
        pending = list(jobs)
        active: list[ServedJob] = []
        peak_active = 0
        peak_bytes = self.ctx.memory_used()
        ticks = 0
        t0 = time.perf_counter()
        ev_start = torch.cuda.Event(enable_timing=True)
        while pending or active:
            now = time.perf_counter() - t0
            while pending and (not real_time or pending[0].arrival <= now) and len(active) < self.max_active:
                if not self._admit(pending[0]):
                    break
                sj = pending.pop(0)
                sj.admitted_at = time.perf_counter() - t0
                active.append(sj)
            if not active:
                if pending and (not real_time or pending[0].arrival <= now):
                    raise RuntimeError(f"job {pending[0].wl.name} does not fit the HBM budget even alone")
                if pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.01)))
                continue
            peak_active = max(peak_active, len(active))
            peak_bytes = max(peak_bytes, self.ctx.memory_used())
            ev_start.record(self.stream)
            if self.mode in ("batched", "graphed"):
                ev_end = torch.cuda.Event(enable_timing=True)
                if self.mode == "graphed":
                    self._graphed_step(active)
                else:
                    api.step_batch(self.ctx, [sj.job for sj in active], stream=self.stream)
                ev_end.record(self.stream)
                ev_end.synchronize()
                dt = ev_start.elapsed_time(ev_end)
                for sj in active:
                    sj.latencies_ms.append(dt)
            else:
                ends = []
                for sj in active:
                    sj.job.step(self.stream)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(self.stream)
                    ends.append(ev)
                ends[-1].synchronize()
                for sj, ev in zip(active, ends):
                    sj.latencies_ms.append(ev_start.elapsed_time(ev))
            ticks += 1
            now = time.perf_counter() - t0
            still = []
            for sj in active:
                sj.done += 1
                if sj.done >= sj.steps:
                    self._retire(sj, now)
                else:
                    still.append(sj)
            active = still
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
        }
        return report, jobs
