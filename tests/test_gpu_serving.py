"""GPU tests of the serving loop and the launch-shape autotuner.

* Continuous batching: jobs arriving while others run are admitted and packed into the
  same launches (also replayed as captured CUDA graphs); every job's final parameters,
  gradient and losses are bit-identical to running it alone (and to the
  one-job-per-launch mode).
* HBM-budget admission: with a budget that fits only a few jobs, the rest wait and are
  admitted as finished jobs free their memory; all complete.
* Admission renders the target on the device (the same image as a host-supplied one), and
  released job blocks are reused without new device memory.
* The autotuner returns one of its candidates and caches it; a job created without a
  launch shape then takes the cached one and runs exactly as a job given that shape
  (the CTA count never changes results; the block shape only regroups FP64 partial sums).
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
    from paper_2211_17263_gb300 import api, capi
    from paper_2211_17263_gb300.serve import Server, admit_job
    arrivals = [(0.0, a[1]) for a in _mix()]
    # measure what each job holds (a budget this small makes the context reserve exactly
    # what each block needs), then allow roughly two at a time
    probe = api.Context(0, hbm_budget_bytes=512 << 20)
    try:
        sizes = []
        side = torch.cuda.Stream()
        for _, wl in arrivals:
            before = probe.memory_used()
            scene, job, ready = admit_job(probe, wl, side)
            ready.synchronize()
            sizes.append(probe.memory_used() - before)
            job.release()
            capi.prdpt_scene_release(probe.handle, scene.id)
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


def test_empty_chunks_are_returned_for_a_larger_job(gpu_lib):
    """Under a budget too small for the arena's 256 MB chunks each block is reserved exactly.
    When a larger job fits neither a free range nor the budget beside the released jobs'
    chunks, the empty chunks go back to the device and the job is admitted."""
    from paper_2211_17263_gb300 import api
    small = workloads.scaled(workloads.config_occlusion(seed=8), width=48, height=40, spp=2, pairs=2)
    big = workloads.scaled(workloads.config_occlusion(seed=8), width=128, height=96, spp=2, pairs=2)

    def held(ctx, wl):  # bytes of the scene's and the job's exact chunks
        before = ctx.memory_used()
        scene = ctx.upload_scene(wl.scene, wl.bindings)
        mid = ctx.memory_used()
        api.Job(scene, wl, None).release()
        return mid - before, ctx.memory_used() - mid

    probe = api.Context(0, hbm_budget_bytes=512 << 20)
    try:
        base = probe.memory_used()
        s_scene, s_small = held(probe, small)
        _, s_big = held(probe, big)  # the big scene is carved from the released small job's chunk
    finally:
        probe.close()
    assert s_big > s_small > 64 * 1024
    budget = base + s_scene + s_small + s_big + 64 * 1024  # slack: the context's descriptor arrays
    ctx = api.Context(0, hbm_budget_bytes=budget)
    try:
        scene = ctx.upload_scene(small.scene, small.bindings)
        th = torch.as_tensor(np.ascontiguousarray(small.theta_ref, np.float32), device="cuda")
        a, b = api.Job(scene, small, None), api.Job(scene, small, None)
        for j in (a, b):
            j.render_target(th)
            j.step()
        a.release()
        b.release()
        torch.cuda.synchronize()
        c = api.Job(scene, big, None)  # refused by the budget unless the two chunks are returned
        c.render_target(th)
        c.step()
        assert c.read()["steps"] == 1
        assert ctx.memory_used() <= budget
        c.release()
    finally:
        ctx.close()


def test_device_rendered_target_equals_host_target(gpu_lib):
    """prdpt_job_render_target renders the same target as prdpt_render_batch: the job's
    trajectory is bit-identical to a job given that image from the host."""
    from paper_2211_17263_gb300 import api
    for wl in (workloads.scaled(workloads.config_occlusion(seed=2), width=40, height=36, spp=4, pairs=3),
               workloads.scaled(workloads.config_gi_box(seed=3), width=24, height=20, spp=2, pairs=2)):
        ctx = api.Context(0)
        try:
            scene = ctx.upload_scene(wl.scene, wl.bindings)
            th = torch.as_tensor(np.ascontiguousarray(wl.theta_ref, np.float32), device="cuda")
            target = scene.render_batch(th[None], wl.width, wl.height, wl.spp, wl.depth, wl.rr_start,
                                        seed=wl.seed, step=0, tag=3, crn=1)[0].cpu().numpy()
            a = api.Job(scene, wl, target)
            b = api.Job(scene, wl, None)
            b.render_target(th)
            for _ in range(4):
                a.step()
                b.step()
            ra, rb = a.read(), b.read()
            for key in ("theta", "grad", "losses"):
                assert np.array_equal(ra[key], rb[key]), (wl.name, key)
            a.release()
            b.release()
        finally:
            ctx.close()


def test_released_blocks_are_reused(gpu_lib):
    """A released job's block returns to the context's arena once its work has completed and
    is carved again for the next job (no new device memory); the new job's results are
    unaffected."""
    from paper_2211_17263_gb300 import api
    wl = workloads.scaled(workloads.config_occlusion(seed=5), width=48, height=40, spp=2, pairs=2)
    ref = api.Context(0)
    try:
        alone = _alone(ref, wl, 3)
    finally:
        ref.close()
    ctx = api.Context(0)
    try:
        scene = ctx.upload_scene(wl.scene, wl.bindings)
        th = torch.as_tensor(np.ascontiguousarray(wl.theta_ref, np.float32), device="cuda")
        first = api.Job(scene, wl, None)
        first.render_target(th)
        for _ in range(5):
            first.step()
        first.release()  # returns at once; the block is in use until the five steps finish
        torch.cuda.synchronize()
        held = ctx.memory_used()
        again = api.Job(scene, wl, None)
        assert ctx.memory_used() == held  # the cached block, not a new allocation
        again.render_target(th)
        for _ in range(3):
            again.step()
        res = again.read()
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(res[key], alone[key]), key
        again.release()
    finally:
        ctx.close()


def test_autotune_picks_and_caches(gpu_lib, tmp_path, monkeypatch):
    from paper_2211_17263_gb300 import api
    from paper_2211_17263_gb300.autotune import CANDIDATES, autotune
    import oracle
    wl = workloads.scaled(workloads.config_occlusion(), width=96, height=64, spp=4, pairs=4)
    target = oracle.render_target(wl)
    cache = str(tmp_path / "tune.json")
    monkeypatch.setenv("PRDPT_AUTOTUNE_CACHE", cache)
    ctx = api.Context(0)
    try:
        scene = ctx.upload_scene(wl.scene, wl.bindings)
        default = api.Job(scene, wl, target)  # empty cache: the library's default shape
        assert default.launch_shape["source"] == "library default"
        best = autotune(scene, wl, target, steps=2)
        assert (best["block_pixels"], best["ctas_per_sm"], best["render_groups"], best["no_path_sharing"]) in CANDIDATES
        assert not best["cached"]
        again = autotune(scene, wl, target)
        assert again["cached"] and again["block_pixels"] == best["block_pixels"]
        # a job created without a launch shape now takes the tuned one, and runs exactly as
        # a job given that shape explicitly
        tuned = api.Job(scene, wl, target)
        assert tuned.launch_shape["source"] == "autotuner cache"
        assert tuned.launch_shape["block_pixels"] == best["block_pixels"]
        explicit = api.Job(scene, wl, target, block_pixels=best["block_pixels"], ctas_per_sm=best["ctas_per_sm"],
                           render_groups=best["render_groups"], no_path_sharing=best["no_path_sharing"],
                           use_tuned=False)
        for j in (tuned, explicit, default):
            for _ in range(2):
                j.step()
        a, b, c = tuned.read(), explicit.read(), default.read()
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(a[key], b[key]), key
        # the CTA count never changes results; the block shape only regroups the FP64 sums
        # of per-block partials, so losses agree to rounding
        assert np.allclose(a["losses"], c["losses"], rtol=1e-6)
        for j in (tuned, explicit, default):
            j.release()
    finally:
        ctx.close()


def test_ctas_per_sm_does_not_change_results(gpu_lib):
    from paper_2211_17263_gb300 import api
    import oracle
    wl = workloads.scaled(workloads.config_caustic(), width=64, height=48, spp=4, pairs=2)
    target = oracle.render_target(wl)
    ctx = api.Context(0)
    try:
        scene = ctx.upload_scene(wl.scene, wl.bindings)
        res = []
        for cps in (1, 2, 0):
            j = api.Job(scene, wl, target, block_pixels=16, ctas_per_sm=cps, use_tuned=False)
            for _ in range(2):
                j.step()
            res.append(j.read())
            j.release()
        for r in res[1:]:
            for key in ("theta", "grad", "losses"):
                assert np.array_equal(r[key], res[0][key]), key
    finally:
        ctx.close()
