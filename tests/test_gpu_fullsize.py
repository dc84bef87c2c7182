"""Parity at the workloads' full sizes, in the launch configuration bench.py times
(automatic pixels-per-item and CTAs-per-SM):

* occlusion (256x256, 16 renders, 16 spp, depth 4) and GI box (512x512, 32 renders,
  32 spp, depth 8 with Russian roulette): the whole gradient and every render's loss
  against the FP64 oracle on the same random streams;
* caustic (512x512, 64 spp, depth 12): 512 sampled pixels of two full renders against
  the oracle's per-pixel paths (the whole 64-render step is too long for the oracle), and
  the gradient of the full image traced in render groups with 8 renders at 64 spp or 64
  renders at 8 spp;
* bandwidth annealing (Sec. 3.3, warm start at half the run): a resident job's
  trajectory against the oracle's schedule.
"""
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


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


@pytest.mark.parametrize("make", [workloads.config_occlusion, workloads.config_gi_box])
def test_full_size_gradient(ctx, make):
    wl = make()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = oracle.render_target(wl)
    opts = scene.grad_opts(wl, step=3)
    g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), opts)
    torch.cuda.synchronize()
    ref = oracle.smoothed_grad(wl, target=target, step=3)
    L = L.cpu().numpy()
    assert np.allclose(L, ref["losses"], rtol=1e-4, atol=1e-9), np.max(np.abs(L / ref["losses"] - 1))
    err = grad_rel_error(g.cpu().numpy(), ref["grad"], ref["weights"], ref["losses"])
    assert err <= GRAD_REL, err


@pytest.mark.parametrize("pairs,spp", [(4, 64), (32, 8)])
def test_full_size_caustic_gradient_shared_and_in_render_groups(ctx, pairs, spp):
    """The caustic image at full size (512x512, depth 12, Russian roulette from vertex 3),
    8 renders at 64 spp and 64 renders at 8 spp: with emitter sharing (each path traced
    once for all renders) and in render groups (every render's paths traced): the gradient
    and every loss against the FP64 oracle, and the two modes bit-identical."""
    wl = workloads.scaled(workloads.config_caustic(), spp=spp, pairs=pairs)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = oracle.render_target(wl)
    ref = oracle.smoothed_grad(wl, target=target, step=2)
    res = {}
    for mode, no_share, paths in (("emit", 0, wl.width * wl.height * wl.spp),
                                  ("groups", 1, wl.renders * wl.width * wl.height * wl.spp)):
        opts = scene.grad_opts(wl, step=2, no_path_sharing=no_share)
        g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), opts)
        torch.cuda.synchronize()
        ctx.counters_enable(True)  # the counting kernel variant, only for its path count
        scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), opts)
        torch.cuda.synchronize()
        assert ctx.counters_read()[3] == paths, mode
        ctx.counters_enable(False)
        L = L.cpu().numpy()
        g = g.cpu().numpy()
        assert np.allclose(L, ref["losses"], rtol=1e-4, atol=1e-9), (mode, np.max(np.abs(L / ref["losses"] - 1)))
        err = grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"])
        assert err <= GRAD_REL, (mode, err)
        res[mode] = (g, L)
    assert np.array_equal(res["emit"][0], res["groups"][0]) and np.array_equal(res["emit"][1], res["groups"][1])


def test_full_size_caustic_sampled_pixels(ctx):
    wl = workloads.config_caustic()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    thetas = np.stack([wl.theta_ref, wl.theta0]).astype(np.float32)
    img = scene.render_batch(_t(thetas), wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, seed=wl.seed,
                             step=1, tag=2, crn=0).cpu().numpy()
    rng = np.random.default_rng(0)
    pix = rng.choice(wl.width * wl.height, size=512, replace=False).astype(np.int32)
    for r in range(2):
        ref = oracle.render_pixels(wl.scene, wl.bindings, thetas[r], pix, wl.width, wl.height, wl.spp, wl.depth,
                                   wl.rr_start, wl.seed, 1, 2, render_field=r)
        gpu = img[r].reshape(-1, 4)[pix, :3]
        diff = np.abs(gpu - ref)
        assert diff.mean() <= 1e-4 and int((diff.max(-1) > 1e-3).sum()) <= 1, (r, diff.mean(), diff.max())


def test_annealed_bandwidth_follows_oracle_schedule(ctx):
    from paper_2211_17263_gb300 import api
    wl = workloads.scaled(workloads.config_small(), width=48, height=48, spp=4, pairs=4)
    wl.anneal, wl.steps, wl.sigma_min = 1, 6, 0.01
    target = oracle.render_target(wl)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    job = api.Job(scene, wl, target)
    th, m, v = wl.theta0.astype(np.float64), np.zeros(wl.D), np.zeros(wl.D)
    for t in range(wl.steps):
        sig = np.array([oracle.sigma_schedule(float(s0), wl.sigma_min, t, wl.steps) for s0 in wl.sigma], np.float32)
        ref = oracle.smoothed_grad(wl, theta=th.astype(np.float32), sigma=sig, target=target, step=t)
        job.step()
        st = job.read()
        assert grad_rel_error(st["grad"], ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL, t
        th, m, v = oracle.adam(th, m, v, ref["grad"], t + 1, wl.lr)
        assert np.allclose(st["theta"], th, rtol=0, atol=2e-5 * (t + 1))
    job.release()
