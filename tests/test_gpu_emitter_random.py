"""Randomised scenes for emitter sharing: every loss and the gradient must equal tracing
one render per work item, bit for bit.

Emitter sharing skips shadow-ray tests against primitives its per-vertex culling deems
out of reach (bounding spheres clear of the cone over the emitter's union bounds, planes
with the vertex and those bounds on one side) and stops shared paths whose rays touch the
union bounds. A culling or touch test that were not conservative would change some
render's next-event estimate or path, so seeded random scenes with occluders near the
lights, mirrors, glass, boxes and two moving emitters (a quad and a sphere with a bound
radius) check both against the per-render kernel.
"""
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


def _random_scene(seed):
    rng = np.random.default_rng(1000 + seed)
    b = workloads.SceneBuilder()
    floor = b.material(workloads.MAT_DIFFUSE, tuple(rng.uniform(0.3, 0.9, 3)))
    b.quad((0, 0, 0), (6, 0, 0), (0, 6, 0), floor)
    if seed % 2:  # a back wall
        b.quad((0, 2.0, 1.5), (6, 0, 0), (0, 0, 3), b.material(workloads.MAT_DIFFUSE, (0.7, 0.6, 0.5)))
    kinds = [workloads.MAT_DIFFUSE, workloads.MAT_MIRROR, workloads.MAT_DIELECTRIC]
    for i in range(3):  # spheres, some of them close under the lights
        m = b.material(kinds[int(rng.integers(0, 3))], tuple(rng.uniform(0.4, 0.95, 3)), ior=1.5)
        c = (float(rng.uniform(-1.2, 1.2)), float(rng.uniform(-1.0, 1.0)), float(rng.uniform(0.3, 1.6)))
        b.sphere(c, float(rng.uniform(0.15, 0.45)), m)
    bm = b.material(workloads.MAT_DIFFUSE, tuple(rng.uniform(0.3, 0.9, 3)))
    b.box((float(rng.uniform(-1, 1)), float(rng.uniform(-1, 1)), 0.3), (0.25, 0.2, 0.3), bm)
    lq = b.material(workloads.MAT_DIFFUSE, (0, 0, 0), emission=(60.0, 60.0, 60.0))
    light = b.quad((float(rng.uniform(-0.5, 0.5)), float(rng.uniform(-0.5, 0.5)), 2.2), (0.4, 0, 0), (0, -0.4, 0), lq)
    lb = b.material(workloads.MAT_DIFFUSE, (0, 0, 0), emission=(20.0, 15.0, 10.0))
    bulb_c = (float(rng.uniform(-1, 1)), float(rng.uniform(-1, 1)), float(rng.uniform(1.2, 1.8)))
    bulb = b.sphere(bulb_c, 0.12, lb)
    b.look_at((0, -4.0, 1.8), (0, 0, 0.6), (0, 0, 1), 45.0)
    wl = workloads.scaled(workloads.config_caustic(seed=seed), width=36, height=28, spp=4, pairs=4)
    wl.scene = b.build()
    lc = wl.scene.prim_geom[light, :3].astype(np.float32)
    binds = [[workloads.BIND_PRIM_POS, light, c] for c in range(3)]
    binds += [[workloads.BIND_PRIM_POS, bulb, c] for c in range(3)]
    binds += [[workloads.BIND_SPHERE_RADIUS, bulb, 0]]
    wl.bindings = np.array(binds, np.int32)
    wl.theta_ref = np.concatenate([lc, np.asarray(bulb_c, np.float32), [0.12]]).astype(np.float32)
    wl.theta0 = (wl.theta_ref + rng.normal(0.0, 0.05, wl.theta_ref.shape)).astype(np.float32)
    wl.sigma = np.full(wl.theta_ref.shape, 0.15, np.float32)
    wl.sigma[-1] = 0.03
    wl.depth, wl.rr_start = 6, 2
    return wl


@pytest.mark.parametrize("seed", range(6))
def test_random_scenes_emitter_sharing_is_bit_identical(ctx, seed):
    wl = _random_scene(seed)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = torch.as_tensor(np.ascontiguousarray(oracle.render_target(wl), np.float32), device="cuda")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")  # noqa: E731
    res = {}
    for key, kw in (("emit", {}), ("per-render", dict(no_path_sharing=1, render_groups=-1))):
        opts = scene.grad_opts(wl, step=seed, block_pixels=8, **kw)
        g, L = scene.smoothed_grad(t(wl.theta0), t(wl.sigma), target, opts)
        torch.cuda.synchronize()
        res[key] = (g.cpu().numpy(), L.cpu().numpy())
    # the mode was in use (the counting kernel variants are separate code: compared only here)
    ctx.counters_enable(True)
    scene.smoothed_grad(t(wl.theta0), t(wl.sigma), target, scene.grad_opts(wl, step=seed, block_pixels=8))
    torch.cuda.synchronize()
    assert ctx.counters_read()[3] == wl.width * wl.height * wl.spp
    ctx.counters_enable(False)
    assert np.array_equal(res["emit"][1], res["per-render"][1]), (seed, res["emit"][1], res["per-render"][1])
    assert np.array_equal(res["emit"][0], res["per-render"][0]), (seed, res["emit"][0], res["per-render"][0])
