"""GPU tests of resident jobs: prdpt_step (sampler + render + Eq. 10 gradient + Adam
on the device) against the oracle's own FP64 trajectory, and packed multi-job
steps (prdpt_step_batch) against each job run alone."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import GRAD_REL, grad_rel_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    from paper_2211_17263_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def _job(ctx, wl, target):
    from paper_2211_17263_gb300 import api
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    return api.Job(scene, wl, target)


def test_job_steps_follow_oracle_trajectory(ctx):
    wl = workloads.config_small()
    target = oracle.render_target(wl)
    job = _job(ctx, wl, target)
    th = wl.theta0.astype(np.float64)
    m = np.zeros(wl.D)
    v = np.zeros(wl.D)
    for t in range(4):
        job.step()
        st = job.read()
        ref = oracle.smoothed_grad(wl, theta=th.astype(np.float32), target=target, step=t)
        assert st["steps"] == t + 1
        assert grad_rel_error(st["grad"], ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL
        assert np.allclose(st["losses"], ref["losses"], rtol=1e-4)
        th, m, v = oracle.adam(th, m, v, ref["grad"], t + 1, wl.lr)
        assert np.allclose(st["theta"], th, rtol=0, atol=2e-5 * (t + 1)), (st["theta"], th)
    job.release()


def test_packed_steps_equal_alone(ctx):
    wls = [workloads.scaled(workloads.config_small(seed=1), width=48, height=40, spp=4, pairs=3),
           workloads.scaled(workloads.config_occlusion(seed=2), width=64, height=64, spp=4, pairs=4),
           workloads.scaled(workloads.config_gi_box(seed=3), width=40, height=32, spp=4, pairs=2)]
    targets = [oracle.render_target(w) for w in wls]
    alone = []
    for w, t in zip(wls, targets):
        j = _job(ctx, w, t)
        for _ in range(3):
            j.step()
        alone.append(j.read())
        j.release()
    from paper_2211_17263_gb300 import api
    jobs = [_job(ctx, w, t) for w, t in zip(wls, targets)]
    for _ in range(3):
        api.step_batch(ctx, jobs)
    for j, a in zip(jobs, alone):
        b = j.read()
        assert b["steps"] == 3
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(a[key], b[key]), key
        j.release()


def test_packed_mixed_sharing_equal_alone(ctx):
    """A batch mixing path-sharing jobs (items = pixel blocks, affected-path and epilogue
    passes) and per-render jobs, listed in interleaved order: the packed step splits them
    into two render launches over one sampler and one finalisation launch; every job
    still matches its own single-job step bit for bit, as do different batch orders."""
    from paper_2211_17263_gb300 import api
    cfgs = [(workloads.config_occlusion(seed=11), 72, 56, 4, 3, 1),  # per-render (sharing off)
            (workloads.config_occlusion(seed=12), 64, 48, 8, 4, 0),  # path sharing
            (workloads.config_gi_box(seed=13), 40, 40, 4, 2, 1),
            (workloads.config_small(seed=14), 56, 40, 4, 2, 0),
            (workloads.config_gi_box(seed=15), 48, 40, 2, 3, 0)]
    wls, flags = [], []
    for wl, w, h, spp, pairs, off in cfgs:
        wls.append(workloads.scaled(wl, width=w, height=h, spp=spp, pairs=pairs))
        flags.append(off)
    targets = [oracle.render_target(w) for w in wls]

    def make(i):
        scene = ctx.upload_scene(wls[i].scene, wls[i].bindings)
        return api.Job(scene, wls[i], targets[i], no_path_sharing=flags[i])

    alone = []
    for i in range(len(wls)):
        j = make(i)
        for _ in range(3):
            j.step()
        alone.append(j.read())
        j.release()
    for order in ([0, 1, 2, 3, 4], [4, 2, 3, 0, 1]):
        jobs = {i: make(i) for i in order}
        for _ in range(3):
            api.step_batch(ctx, [jobs[i] for i in order])
        for i in order:
            b = jobs[i].read()
            assert b["steps"] == 3
            for key in ("theta", "grad", "losses"):
                assert np.array_equal(alone[i][key], b[key]), (order, i, key)
            jobs[i].release()


def test_packed_four_kinds_equal_alone(ctx):
    """A batch with emitter-sharing jobs, path-sharing jobs, render-group jobs and
    one-render-per-item jobs: the packed step runs one render launch per kind; every job
    matches its single-job step."""
    from paper_2211_17263_gb300 import api
    cfgs = [(workloads.config_caustic(seed=51), 40, 32, 2, 8, 0, 1),   # render groups of 16
            (workloads.config_occlusion(seed=52), 48, 40, 4, 3, 0, 0),  # path sharing
            (workloads.config_gi_box(seed=53), 40, 32, 2, 4, -1, 0),    # one render per item
            (workloads.config_gi_box(seed=54), 32, 24, 2, 2, 0, 0),     # render groups of 4
            (workloads.config_caustic(seed=55), 36, 28, 3, 6, 0, 0)]    # emitter sharing
    wls = [workloads.scaled(wl, width=w, height=h, spp=spp, pairs=p) for wl, w, h, spp, p, _, _ in cfgs]
    groups = [c[5] for c in cfgs]
    no_share = [c[6] for c in cfgs]
    targets = [oracle.render_target(w) for w in wls]

    def make(i):
        scene = ctx.upload_scene(wls[i].scene, wls[i].bindings)
        return api.Job(scene, wls[i], targets[i], render_groups=groups[i], no_path_sharing=no_share[i],
                       use_tuned=False)

    alone = []
    for i in range(len(wls)):
        j = make(i)
        for _ in range(2):
            j.step()
        alone.append(j.read())
        j.release()
    order = [3, 0, 4, 2, 1]
    jobs = {i: make(i) for i in order}
    for _ in range(2):
        api.step_batch(ctx, [jobs[i] for i in order])
    for i in order:
        b = jobs[i].read()
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(alone[i][key], b[key]), (i, key)
        jobs[i].release()


def test_packed_emitter_sharing_jobs_of_different_shapes_equal_alone(ctx):
    """Emitter-sharing jobs of different render counts, images and scenes packed into one
    launch: the kernel's CTAs restage the job, scene, per-render records and union bounds
    whenever their next block belongs to another job; every job matches its single-job step."""
    from paper_2211_17263_gb300 import api
    wls = [workloads.scaled(workloads.config_caustic(seed=61), width=40, height=32, spp=3, pairs=3),
           workloads.scaled(workloads.config_caustic(seed=62), width=24, height=24, spp=2, pairs=32),
           workloads.scaled(workloads.config_caustic(seed=63), width=32, height=20, spp=5, pairs=12)]
    targets = [oracle.render_target(w) for w in wls]

    def make(i):
        scene = ctx.upload_scene(wls[i].scene, wls[i].bindings)
        return api.Job(scene, wls[i], targets[i], block_pixels=8, use_tuned=False)

    alone = []
    for i in range(len(wls)):
        j = make(i)
        for _ in range(2):
            j.step()
        alone.append(j.read())
        j.release()
    jobs = [make(i) for i in (2, 0, 1)]
    for _ in range(2):
        api.step_batch(ctx, jobs)
    for i, j in zip((2, 0, 1), jobs):
        b = j.read()
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(alone[i][key], b[key]), (i, key)
        j.release()


def test_job_release_and_reuse_of_batch(ctx):
    from paper_2211_17263_gb300 import api
    wl = workloads.scaled(workloads.config_small(), width=16, height=16, spp=1, pairs=1)
    target = oracle.render_target(wl)
    a, b = _job(ctx, wl, target), _job(ctx, wl, target)
    api.step_batch(ctx, [a, b])
    a.release()
    api.step_batch(ctx, [b])
    assert b.read()["steps"] == 2
    b.release()


def test_alternating_batches_on_a_side_stream(ctx):
    """Packed steps of two different job sets, alternating on a non-blocking stream with no
    host synchronisation in between: each change of set uploads new job descriptors, in
    stream order, so the steps still in flight keep theirs. Every job ends where it ends
    when it steps alone."""
    from paper_2211_17263_gb300 import api
    wls = [workloads.scaled(workloads.config_small(seed=21), width=48, height=40, spp=4, pairs=3),
           workloads.scaled(workloads.config_occlusion(seed=22), width=64, height=48, spp=4, pairs=4),
           workloads.scaled(workloads.config_gi_box(seed=23), width=40, height=32, spp=2, pairs=2)]
    targets = [oracle.render_target(w) for w in wls]
    steps = [4, 8, 4]  # job 1 is in both sets
    alone = []
    for w, t, n in zip(wls, targets, steps):
        j = _job(ctx, w, t)
        for _ in range(n):
            j.step()
        alone.append(j.read())
        j.release()
    jobs = [_job(ctx, w, t) for w, t in zip(wls, targets)]
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(4):
        api.step_batch(ctx, [jobs[0], jobs[1]], stream=side)
        api.step_batch(ctx, [jobs[1], jobs[2]], stream=side)
    side.synchronize()
    for j, a, n in zip(jobs, alone, steps):
        b = j.read()
        assert b["steps"] == n
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(a[key], b[key]), key
        j.release()


def test_jobs_step_concurrently_on_their_own_streams(ctx):
    """Resident jobs own their buffers: two jobs (one sharing paths, one not) stepping
    on two streams at once end exactly where they end stepping alone."""
    from paper_2211_17263_gb300 import api
    wls = [workloads.scaled(workloads.config_occlusion(seed=31), width=64, height=48, spp=4, pairs=4),
           workloads.scaled(workloads.config_gi_box(seed=32), width=48, height=40, spp=2, pairs=2)]
    targets = [oracle.render_target(w) for w in wls]
    alone = []
    for w, t in zip(wls, targets):
        j = _job(ctx, w, t)
        for _ in range(5):
            j.step()
        alone.append(j.read())
        j.release()
    jobs = [_job(ctx, w, t) for w, t in zip(wls, targets)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for _ in range(5):
        for j, s in zip(jobs, streams):
            j.step(s)
    for s in streams:
        s.synchronize()
    for j, a in zip(jobs, alone):
        b = j.read()
        assert b["steps"] == 5
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(a[key], b[key]), key
        j.release()


def test_jobs_step_from_several_host_threads(ctx):
    """Two host threads step two jobs on their own streams while a third creates, reads
    and releases jobs on the same context: the stepped jobs end exactly where they end
    stepping alone."""
    import threading
    wls = [workloads.scaled(workloads.config_occlusion(seed=41), width=48, height=40, spp=4, pairs=4),
           workloads.scaled(workloads.config_small(seed=42), width=40, height=32, spp=4, pairs=4)]
    targets = [oracle.render_target(w) for w in wls]
    alone = []
    for w, t in zip(wls, targets):
        j = _job(ctx, w, t)
        for _ in range(20):
            j.step()
        alone.append(j.read())
        j.release()
    jobs = [_job(ctx, w, t) for w, t in zip(wls, targets)]
    torch.cuda.synchronize()
    errors = []

    def stepper(j):
        try:
            s = torch.cuda.Stream()
            for _ in range(20):
                j.step(s)
            s.synchronize()
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    def churn():
        try:
            for _ in range(5):
                j = _job(ctx, wls[1], targets[1])
                j.read()
                j.release()
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    threads = [threading.Thread(target=stepper, args=(j,)) for j in jobs] + [threading.Thread(target=churn)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for j, a in zip(jobs, alone):
        b = j.read()
        assert b["steps"] == 20
        for key in ("theta", "grad", "losses"):
            assert np.array_equal(a[key], b[key]), key
        j.release()


def test_too_many_work_items_is_an_argument_error(ctx):
    """The render kernels number (render, pixel block) work items with 32-bit integers: a
    job of 512 renders of 8192^2 pixels in 8-pixel blocks (4.3 G items) is refused with an
    argument error before anything is allocated or read."""
    from paper_2211_17263_gb300 import api, capi
    wl = workloads.config_occlusion()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    small = np.zeros(16, np.float32)  # never read: the call fails before the uploads
    opts = scene.grad_opts(wl, pairs=256, block_pixels=8, no_path_sharing=1)
    opts.width = opts.height = 8192
    desc = capi.prdpt_job_desc(grad=opts, theta0_host=small.ctypes.data, sigma0_host=small.ctypes.data,
                               target_host=small.ctypes.data, lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8,
                               sigma_min=0.01, anneal=0, total_steps=1)
    before = ctx.memory_used()
    with pytest.raises(capi.PrdptError, match="work items"):
        capi.prdpt_job_create(ctx.handle, scene.id, desc)
    assert ctx.memory_used() == before
