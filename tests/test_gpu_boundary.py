"""The C ABI at its limits: degenerate and out-of-range arguments are refused with the
documented status before anything is launched (and the context stays usable), and the
largest pair count, the widest image strip and the deepest paths the header allows
still agree with the FP64 oracle."""
import copy
import math

import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import GRAD_REL, grad_rel_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

INVALID_ARG, NOT_FOUND = 1, 6


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    from paper_2211_17263_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def _ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def test_invalid_arguments_are_refused_and_the_context_survives(ctx):
    from paper_2211_17263_gb300 import capi
    wl = workloads.scaled(workloads.config_occlusion(), width=24, height=16, spp=2, pairs=2)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = _t(oracle.render_target(wl))
    theta, sigma = _t(wl.theta0), _t(wl.sigma)
    good = scene.grad_opts(wl, step=1)
    g0, L0 = scene.smoothed_grad(theta, sigma, target, good)
    g0, L0 = g0.cpu().numpy(), L0.cpu().numpy()
    bad = {"pairs": [0, 257], "width": [0, 8193], "height": [0, -1], "spp": [0, 65536], "depth": [0, 65],
           "rr_start": [-2, 65], "sampler": [-1, 3], "estimator": [2], "pair_begin": [-1, (1 << 26) + 1]}
    grad, losses = torch.empty(wl.D, device="cuda"), torch.empty(2 * 257, device="cuda")
    for field, values in bad.items():
        for v in values:
            o = copy.copy(good)
            setattr(o, field, v)
            with pytest.raises(capi.PrdptError) as e:
                capi.prdpt_smoothed_grad(ctx.handle, scene.id, _ptr(theta), _ptr(sigma), o, _ptr(target),
                                         _ptr(grad), _ptr(losses), None)
            assert e.value.code == INVALID_ARG, (field, v)
    with pytest.raises(capi.PrdptError) as e:  # a NULL buffer
        capi.prdpt_smoothed_grad(ctx.handle, scene.id, _ptr(theta), _ptr(sigma), good, None, _ptr(grad),
                                 _ptr(losses), None)
    assert e.value.code == INVALID_ARG
    with pytest.raises(capi.PrdptError) as e:  # an unknown scene
        capi.prdpt_smoothed_grad(ctx.handle, 1 << 20, _ptr(theta), _ptr(sigma), good, _ptr(target), _ptr(grad),
                                 _ptr(losses), None)
    assert e.value.code == NOT_FOUND
    with pytest.raises(capi.PrdptError) as e:  # an empty render batch
        scene.render_batch(theta[None][:0], 8, 8, 1, 1)
    assert e.value.code == INVALID_ARG
    th, m, v = (np.ascontiguousarray(a, np.float32) for a in (wl.theta0, np.zeros(wl.D), np.zeros(wl.D)))
    with pytest.raises(capi.PrdptError) as e:  # Adam's step counts from 1
        scene.step_host(th, m, v, 0, wl.lr, np.ascontiguousarray(wl.sigma, np.float32),
                        np.ascontiguousarray(target.cpu().numpy()), good)
    assert e.value.code == INVALID_ARG
    assert np.array_equal(th, wl.theta0.astype(np.float32)) and not m.any() and not v.any()  # left untouched
    g1, L1 = scene.smoothed_grad(theta, sigma, target, good)  # nothing refused left a trace
    assert np.array_equal(g1.cpu().numpy(), g0) and np.array_equal(L1.cpu().numpy(), L0)


def _grad_vs_oracle(ctx, wl, step):
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = oracle.render_target(wl)
    g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), scene.grad_opts(wl, step=step))
    torch.cuda.synchronize()
    ref = oracle.smoothed_grad(wl, target=target, step=step)
    return g.cpu().numpy(), L.cpu().numpy(), ref


def test_maximum_pair_count_matches_oracle(ctx):
    """P = 256 antithetic pairs (512 renders), the most one call takes."""
    wl = workloads.scaled(workloads.config_occlusion(), width=16, height=12, spp=2, pairs=256)
    g, L, ref = _grad_vs_oracle(ctx, wl, step=4)
    assert L.shape == (512,)
    assert np.allclose(L, ref["losses"], rtol=1e-4, atol=1e-9)
    assert grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL


def test_widest_strip_matches_oracle(ctx):
    """An 8192 x 1 image: the largest width, one row (every pixel block ragged), through
    the box at theta0 with a 60-degree horizontal field of view."""
    wl = workloads.scaled(workloads.config_occlusion(), width=8192, height=1, spp=1, pairs=2)
    wl.scene.camera[3:6] = wl.theta0  # look at the box
    wl.scene.camera[9] = math.degrees(2.0 * math.atan(math.tan(math.radians(30.0)) / 8192.0))  # vertical fov
    g, L, ref = _grad_vs_oracle(ctx, wl, step=0)
    assert np.abs(ref["grad"]).max() > 1e-3  # the strip sees the box move
    assert np.allclose(L, ref["losses"], rtol=1e-4, atol=1e-9)
    assert grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL


def test_deepest_paths_match_oracle(ctx):
    """depth 64 (the largest) without Russian roulette in the diffuse GI box."""
    wl = workloads.scaled(workloads.config_gi_box(), width=24, height=24, spp=2, depth=64, rr_start=-1)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    thetas = np.stack([wl.theta_ref, wl.theta0]).astype(np.float32)
    img = scene.render_batch(_t(thetas), wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, seed=wl.seed, step=1,
                             tag=2, crn=1).cpu().numpy()
    ref = oracle.render(wl.scene, wl.bindings, thetas, wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, wl.seed,
                        1, 2, 1)
    diff = np.abs(img[..., :3] - ref)
    assert diff.mean() <= 1e-4 and (diff.max(-1) > 1e-3).sum() <= max(1, int(1e-3 * diff[..., 0].size))
