"""GPU parity of the pathwise estimator (Eq. 9, kappa-dP) against the FP64 oracle on the
same draws and path samples: per-render losses and the mean of the renders' pathwise
loss gradients, for albedo and emission parameters (depth 1 and multi-bounce with
Russian roulette, ragged image blocks, 4-, 6- and 8-slot tangent kernels), a resident job's
trajectory, and the argument checks."""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import GRAD_REL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = GRAD_REL       # gradient: ||g_gpu - g_orc|| / ||g_orc|| (these gradients are far from zero)
LOSS_RTOL = 1e-4     # per-render losses


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    from paper_2211_17263_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def _cases():
    small = workloads.config_small_albedo
    gi = workloads.config_gi_albedo
    return {
        "small-d1": lambda: workloads.scaled(small(), width=40, height=29, spp=4, pairs=3),
        "small-d3-rr": lambda: workloads.scaled(small(), width=33, height=20, spp=4, pairs=2, depth=3, rr_start=1),
        "small-4-params": lambda: _subset(workloads.scaled(small(), width=24, height=24, spp=2, pairs=2), 4),
        "gi-walls": lambda: workloads.scaled(gi(), width=48, height=37, spp=4, pairs=2),
        "gi-8-params": lambda: _with_back_wall_rg(workloads.scaled(gi(), width=40, height=32, spp=4, pairs=2)),
    }


def _with_back_wall_rg(wl):
    """Eight parameters (the 8-slot tangent kernel): the two side walls' RGB and material 0's
    red and green albedo."""
    m = 0
    extra = np.array([[workloads.BIND_MAT_ALBEDO, m, 0], [workloads.BIND_MAT_ALBEDO, m, 1]], np.int32)
    base = wl.scene.mat_param[m, :2].astype(np.float32)
    wl.bindings = np.vstack([wl.bindings, extra]).astype(np.int32)
    wl.theta_ref = np.append(wl.theta_ref, base).astype(np.float32)
    wl.theta0 = np.append(wl.theta0, base + np.float32(0.1)).astype(np.float32)
    wl.sigma = np.append(wl.sigma, np.full(2, 0.125, np.float32)).astype(np.float32)
    return wl


def _subset(wl, n):
    wl.bindings, wl.theta_ref, wl.theta0, wl.sigma = (wl.bindings[:n].copy(), wl.theta_ref[:n].copy(),
                                                      wl.theta0[:n].copy(), wl.sigma[:n].copy())
    return wl


def _gpu_grad(ctx, wl, target, step=0):
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    opts = scene.grad_opts(wl, step=step)
    g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), opts)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64), L.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", list(_cases()))
def test_pathwise_gradient_matches_oracle(ctx, case):
    wl = _cases()[case]()
    target = oracle.render_target(wl)
    g, L = _gpu_grad(ctx, wl, target, step=2)
    ref = oracle.kdp_grad(wl, target=target, step=2)
    assert np.allclose(L, ref["losses"], rtol=LOSS_RTOL), (L, ref["losses"])
    err = np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"])
    assert err <= REL, (case, g, ref["grad"], err)


def test_pathwise_gradient_full_size_gi(ctx):
    """The GI box at full size (512 x 512, depth 8, 32 spp, Russian roulette) with two
    pairs, in the launch configuration of a resident step."""
    wl = workloads.scaled(workloads.config_gi_albedo(), pairs=2)
    target = oracle.render_target(wl)
    g, L = _gpu_grad(ctx, wl, target, step=1)
    ref = oracle.kdp_grad(wl, target=target, step=1)
    assert np.allclose(L, ref["losses"], rtol=LOSS_RTOL)
    assert np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"]) <= REL


def test_pathwise_job_follows_oracle_trajectory(ctx):
    from paper_2211_17263_gb300 import api
    wl = workloads.scaled(workloads.config_small_albedo(), width=32, height=24, spp=4, pairs=2)
    target = oracle.render_target(wl)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    job = api.Job(scene, wl, target)
    th = wl.theta0.astype(np.float64)
    m = np.zeros(wl.D)
    v = np.zeros(wl.D)
    for t in range(3):
        job.step()
        st = job.read()
        ref = oracle.kdp_grad(wl, theta=th.astype(np.float32), target=target, step=t)
        assert np.linalg.norm(st["grad"] - ref["grad"]) / np.linalg.norm(ref["grad"]) <= REL
        assert np.allclose(st["losses"], ref["losses"], rtol=LOSS_RTOL)
        th, m, v = oracle.adam(th, m, v, ref["grad"], t + 1, wl.lr)
        assert np.allclose(st["theta"], th, rtol=1e-5, atol=2e-5 * (t + 1)), (st["theta"], th)
    job.release()


def test_pathwise_argument_checks(ctx):
    from paper_2211_17263_gb300 import api, capi
    geo = workloads.scaled(workloads.config_small(), width=8, height=8, spp=1, pairs=1)
    geo.sampler, geo.estimator = workloads.SAMPLER_GAUSS, 1
    target = np.zeros((8, 8, 4), np.float32)
    scene = ctx.upload_scene(geo.scene, geo.bindings)
    with pytest.raises(capi.PrdptError):  # geometry bindings have no pathwise derivative here
        scene.smoothed_grad(_t(geo.theta0), _t(geo.sigma), _t(target), scene.grad_opts(geo))
    mat = workloads.scaled(workloads.config_small_albedo(), width=8, height=8, spp=1, pairs=1)
    scene2 = ctx.upload_scene(mat.scene, mat.bindings)
    with pytest.raises(capi.PrdptError):  # the kernel must be sampled exactly: Gaussian draws
        scene2.smoothed_grad(_t(mat.theta0), _t(mat.sigma), _t(target),
                             scene2.grad_opts(mat, sampler=workloads.SAMPLER_RADIAL))
    a = api.Job(scene2, mat, target)
    b = api.Job(scene2, mat, target)
    with pytest.raises(capi.PrdptError):  # pathwise jobs step alone
        api.step_batch(ctx, [a, b])
    a.release()
    b.release()
