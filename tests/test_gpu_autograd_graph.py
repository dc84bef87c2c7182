"""GPU tests of the autograd Function and of CUDA-graph capture of resident steps.

* SmoothedLoss.backward (the Eq. 10 estimator) against central finite differences
  (h = 1e-3) of the Gaussian-smoothed objective, both on the same path-sample streams:
  the smoothed objective of step t is E_z L(theta + sigma z; paths of step t), estimated
  with K Gaussian draws z rendered by the library's forward renderer; the estimator is
  averaged over the same steps. Pass: |mean g - FD| <= 4.5 combined standard errors.
* torch.optim.Adam driven by SmoothedLoss follows the resident job's on-device Adam.
* 300 resident steps captured in one CUDA graph give bit-identical parameters to 300
  eagerly launched steps.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

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


def _mse(imgs, target):
    return ((imgs[..., :3] - target[None, ..., :3]).double() ** 2).mean(dim=(1, 2, 3))


def test_backward_matches_fd_of_smoothed_objective(ctx):
    from paper_2211_17263_gb300.autograd import SmoothedLoss
    wl = workloads.scaled(workloads.config_occlusion(), width=96, height=96, spp=4, pairs=8)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = _t(oracle.render_target(wl))
    sigma = _t(wl.sigma)
    M = 64  # optimiser steps (path-sample sets) averaged over
    gs = []
    for t in range(M):
        theta = _t(wl.theta0).requires_grad_(True)
        loss = SmoothedLoss.apply(theta, scene, sigma, target, scene.grad_opts(wl, step=t))
        loss.backward()
        gs.append(theta.grad.detach().cpu().numpy().astype(np.float64))
    gs = np.array(gs)
    g_mean, g_se = gs.mean(0), gs.std(0, ddof=1) / math.sqrt(M)

    K_per_step, h = 64, 1e-3
    rng = np.random.default_rng(7)
    fd_samples = []
    for t in range(M):
        z = rng.normal(size=(K_per_step, wl.D)).astype(np.float64)
        base = wl.theta0.astype(np.float64)[None, :] + z * wl.sigma.astype(np.float64)[None, :]
        per_d = []
        for d in range(wl.D):
            e = np.zeros(wl.D)
            e[d] = h
            th = np.concatenate([base + e, base - e]).astype(np.float32)
            imgs = scene.render_batch(_t(th), wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, seed=wl.seed,
                                      step=t, tag=2, crn=1)
            L = _mse(imgs, target).cpu().numpy()
            per_d.append((L[:K_per_step] - L[K_per_step:]) / (2 * h))
        fd_samples.append(np.stack(per_d, 1))
    fd_samples = np.concatenate(fd_samples)
    fd_mean = fd_samples.mean(0)
    fd_se = fd_samples.std(0, ddof=1) / math.sqrt(fd_samples.shape[0])
    se = np.sqrt(g_se ** 2 + fd_se ** 2)
    assert np.all(np.abs(g_mean - fd_mean) <= 4.5 * se), (g_mean, fd_mean, se)
    big = np.argmax(np.abs(fd_mean))
    assert se[big] < 0.5 * abs(fd_mean[big]), (fd_mean, se)  # the comparison has power


def test_torch_adam_on_autograd_matches_resident_job(ctx):
    from paper_2211_17263_gb300 import api
    from paper_2211_17263_gb300.autograd import SmoothedLoss
    wl = workloads.scaled(workloads.config_small(), width=48, height=48, spp=4, pairs=4)
    target_np = oracle.render_target(wl)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target, sigma = _t(target_np), _t(wl.sigma)
    theta = torch.nn.Parameter(_t(wl.theta0))
    opt = torch.optim.Adam([theta], lr=wl.lr, betas=(0.9, 0.999), eps=1e-8)
    for t in range(5):
        opt.zero_grad()
        SmoothedLoss.apply(theta, scene, sigma, target, scene.grad_opts(wl, step=t)).backward()
        opt.step()
    job = api.Job(scene, wl, target_np)
    for _ in range(5):
        job.step()
    st = job.read()
    job.release()
    assert st["steps"] == 5
    assert np.allclose(theta.detach().cpu().numpy(), st["theta"], rtol=0, atol=1e-5)


@pytest.mark.parametrize("make", [
    lambda: workloads.scaled(workloads.config_gi_box(), width=32, height=24, spp=2, pairs=2),  # render groups
    lambda: workloads.scaled(workloads.config_caustic(), width=32, height=24, spp=4, pairs=4),  # emitter sharing
])
def test_cuda_graph_of_300_steps_is_bit_identical(ctx, make):
    from paper_2211_17263_gb300 import api
    wl = make()
    target = oracle.render_target(wl)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    eager = api.Job(scene, wl, target)
    graphed = api.Job(scene, wl, target)
    n = 300
    for _ in range(n):
        eager.step()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        for _ in range(n):
            graphed.step()
    g.replay()
    torch.cuda.synchronize()
    a, b = eager.read(), graphed.read()
    assert a["steps"] == n and b["steps"] == n
    for key in ("theta", "grad", "losses"):
        assert np.array_equal(a[key], b[key]), key
    eager.release()
    graphed.release()
