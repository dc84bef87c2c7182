"""GPU parity of the high-dimensional parameter path (texture scenes) against the FP64
oracle: texel lookup in the render, the D-dimensional draws of every sampler, the
gradient g = W^T dL / 2P over the texels, a resident job's Adam trajectory, and the
49,152-parameter texture at full size."""
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


def test_texture_render_matches_oracle(ctx):
    wl = workloads.config_texture(res=16, px_per_texel=2)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    assert scene.D == 768
    thetas = np.stack([wl.theta_ref, wl.theta_ref * 2.5 - 0.75])  # the second clamps at 0 and 1
    imgs = scene.render_batch(_t(thetas), wl.width, wl.height, 3, wl.depth, wl.rr_start, seed=1, step=0, tag=2,
                              crn=1).cpu().numpy()[..., :3]
    ref = oracle.render(wl.scene, wl.bindings, thetas, wl.width, wl.height, 3, wl.depth, seed=1)
    assert np.abs(imgs - ref).max() < 1e-6


@pytest.mark.parametrize("sampler", [0, 1, 2])
def test_texture_draws_match_oracle(ctx, sampler):
    D, pairs = 3 * 24 * 24, 3
    sigma = np.full(D, 0.02, np.float32)
    sigma[::7] = 0.05
    tau, w = ctx.sample_perturbations(_t(sigma), pairs, sampler=sampler, antithetic=1, seed=77, step=4)
    tau, w = tau.cpu().numpy(), w.cpu().numpy()
    for p in range(pairs):
        t64, _, w64 = oracle.sample(sampler, sigma, seed=77, step=4, index=p)
        np.testing.assert_allclose(tau[2 * p], t64, rtol=2e-5, atol=1e-9)
        np.testing.assert_allclose(w[2 * p], w64, rtol=2e-5, atol=1e-6)
        assert np.array_equal(tau[2 * p + 1], -tau[2 * p]) and np.array_equal(w[2 * p + 1], -w[2 * p])


def _grad_case(ctx, wl, step=0):
    target = oracle.render_target(wl)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), scene.grad_opts(wl, step=step))
    torch.cuda.synchronize()
    ref = oracle.smoothed_grad(wl, target=target, step=step)
    return g.cpu().numpy().astype(np.float64), L.cpu().numpy().astype(np.float64), ref


@pytest.mark.parametrize("res,px", [(16, 2), (12, 3)])
def test_texture_gradient_matches_oracle(ctx, res, px):
    wl = workloads.config_texture(res=res, px_per_texel=px)
    wl.pairs, wl.spp = 4, 2
    g, L, ref = _grad_case(ctx, wl, step=2)
    assert np.allclose(L, ref["losses"], rtol=1e-5)
    assert grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL


def test_texture_gradient_full_size(ctx):
    """The 128 x 128 RGB texture (49,152 parameters) at its full render size."""
    wl = workloads.config_texture()
    assert wl.D == 49152
    g, L, ref = _grad_case(ctx, wl, step=1)
    assert np.allclose(L, ref["losses"], rtol=1e-5)
    assert grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL


def test_texture_job_follows_oracle_trajectory(ctx):
    from paper_2211_17263_gb300 import api, capi
    wl = workloads.config_texture(res=8, px_per_texel=2)
    wl.pairs = 3
    target = oracle.render_target(wl)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    before = ctx.memory_used()
    job = api.Job(scene, wl, target)
    th = wl.theta0.astype(np.float64)
    m = np.zeros(wl.D)
    v = np.zeros(wl.D)
    for t in range(3):
        job.step()
        st = job.read()
        ref = oracle.smoothed_grad(wl, theta=th.astype(np.float32), target=target, step=t)
        assert grad_rel_error(st["grad"], ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL
        th, m, v = oracle.adam(th, m, v, ref["grad"], t + 1, wl.lr)
        assert np.allclose(st["theta"], th, rtol=0, atol=2e-5 * (t + 1))
    other = api.Job(scene, wl, target)
    with pytest.raises(capi.PrdptError):  # texture jobs step alone
        api.step_batch(ctx, [job, other])
    job.release()
    other.release()
    torch.cuda.synchronize()
    held = ctx.memory_used()  # the released jobs' blocks are kept for reuse
    assert held >= before
    again = api.Job(scene, wl, target)  # takes a cached block: no new device memory
    assert ctx.memory_used() == held
    again.release()
