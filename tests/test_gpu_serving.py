"""GPU tests of the serving loop and the launch-shape autotuner.

* Continuous batching: jobs arriving while others run are admitted and packed into the
  same launches (also replayed as captured CUDA graphs); every job's final parameters,
  gradient and losses are bit-identical to running it alone (and to the
  one-job-per-launch mode).
* HBM-budget admission: with a budget that fits only a few jobs, the rest wait and are
  admitted as finished jobs free their memory; all complete.
* The autotuner returns one of its candidates, caches it, and the tuned launch gives the
  same losses as the default launch (block shape only regroups FP64 partial sums).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mix():
    base = [workloads.config_small(seed=3), workloads.config_occlusion(seed=4), workloads.config_gi_box(seed=5),
            workloads.config_small(seed=6), workloads.config_occlusion(seed=7)]
    sizes = [(40, 32, 2, 2, 60), (48, 40, 2, 3, 50), (32, 24, 2, 2, 70), (24, 24, 4, 1, 40), (56, 48, 1, 2, 60)]
    out = []
    for i, (wl, (w, h, spp, pairs, steps)) in enumerate(zip(base, sizes)):
        s = workloads.scaled(wl, width=w, height=h, spp=spp, pairs=pairs)
        s.steps = steps
        out.append((0.0005 * i, s))  # later jobs arrive while the first ones are running
    return out


def _alone(ctx, wl, steps):
    from paper_2211_17263_gb300 import api, capi
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    th = torch.as_tensor(np.ascontiguousarray(wl.theta_ref[None], np.float32), device="cuda")
    target = scene.render_batch(th, wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, seed=wl.seed, step=0,
                                tag=3, crn=1)[0].cpu().numpy()
    job = api.Job(scene, wl, target)
    for _ in range(steps):
        job.step()
    res = job.read()
    job.release()
    capi.prdpt_scene_release(ctx.handle, scene.id)
    return res


@pytest.mark.parametrize("mode", ["batched", "graphed", "plain"])
def test_served_results_equal_alone(gpu_lib, mode):
    from paper_2211_17263_gb300 import api
    from paper_2211_17263_gb300.serve import Server
    ctx = api.Context(0)
    try:
        report, jobs = Server(ctx, mode=mode).run(_mix(), real_time=True)
        assert report["jobs"] == 5 and report["job_steps"] == sum(j.steps for j in jobs)
        assert report["p50_ms"] > 0 and report["p99_ms"] >= report["p50_ms"]
        for sj in jobs:
            alone = _alone(ctx, sj.wl, sj.steps)
            assert sj.result["steps"] == sj.steps == alone["steps"]
            for key in ("theta", "grad", "losses"):
                assert np.array_equal(sj.result[key], alone[key]), (mode, sj.wl.name, key)
        if mode != "plain":
            assert report["peak_active"] >= 2  # arrivals overlapped on the device
        if mode == "graphed":
            assert report["graph_replays"] > 0  # stable stretches ran as graph replays
    finally:
        ctx.close()


def test_budget_limits_admission(gpu_lib):
    from paper_2211_17263_gb300 import api
    from paper_2211_17263_gb300.serve import Server
    arrivals = [(0.0, a[1]) for a in _mix()]
    probe = api.Context(0)  # measure what each job holds, then allow roughly two at a time
    try:
        sizes, before = [], probe.memory_used()
        for _, wl in arrivals:
            _alone(probe, wl, 1)
        srv = Server(probe, mode="batched")
        for _, wl in arrivals:
            from paper_2211_17263_gb300.serve import ServedJob
            sj = ServedJob(wl=wl, arrival=0.0, steps=1)
            srv._admit(sj)
            sizes.append(probe.memory_used() - before)
            srv._retire(sj, 0.0)
    finally:
        probe.close()
    budget = 2 * max(sizes) + 64 * 1024  # plus the context's own scratch (control words, descriptors)
    ctx = api.Context(0, hbm_budget_bytes=budget)
    try:
        report, jobs = Server(ctx, mode="batched").run(arrivals, real_time=False)
        assert all(sj.result is not None and sj.result["steps"] == sj.steps for sj in jobs)
        assert report["peak_active"] < len(jobs)
    finally:
        ctx.close()


def test_autotune_picks_and_caches(gpu_lib, tmp_path):
    from paper_2211_17263_gb300 import api
    from paper_2211_17263_gb300.autotune import CANDIDATES, autotune
    import oracle
    wl = workloads.scaled(workloads.config_occlusion(), width=96, height=64, spp=4, pairs=4)
    target = oracle.render_target(wl)
    ctx = api.Context(0)
    try:
        scene = ctx.upload_scene(wl.scene, wl.bindings)
        cache = str(tmp_path / "tune.json")
        best = autotune(scene, wl, target, cache_path=cache, steps=2)
        assert (best["block_pixels"], best["ctas_per_sm"]) in CANDIDATES and not best["cached"]
        again = autotune(scene, wl, target, cache_path=cache)
        assert again["cached"] and again["block_pixels"] == best["block_pixels"]
        tuned = api.Job(scene, wl, target, block_pixels=best["block_pixels"], ctas_per_sm=best["ctas_per_sm"])
        default = api.Job(scene, wl, target)
        tuned.step()
        default.step()
        a, b = tuned.read(), default.read()
        assert np.allclose(a["losses"], b["losses"], rtol=1e-6)
        tuned.release()
        default.release()
    finally:
        ctx.close()
