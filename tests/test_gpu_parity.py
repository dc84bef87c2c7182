"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the
same seeded inputs and the same Philox streams.

* Philox words: bit-exact.
* Perturbations tau and weights w (Sec. 3.2, Eq. 11): the oracle's FP64 values
  rounded to FP32, within a few FP32 ulps (CUDA's logf / sqrtf / sincospif error
  bounds are 1-2 ulp).
* Images (Eq. 3): mean abs error <= 1e-4 and <= 0.1 % outlier pixels (> 1e-3).
* Gradient (Eq. 10): relative error <= 1e-3; per-render losses to 1e-4 relative.
"""
import numpy as np
import pytest

import oracle
import workloads
from gpu_helpers import GRAD_REL, assert_image_parity, grad_rel_error

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


# ---------------------------------------------------------------- random streams
@pytest.mark.parametrize("c1,c2,c3", [(0, 0, 0), (5 | (3 << 16) | (1 << 24), 17, (2 << 28) | 9),
                                      (0xFFFF, 0xFFFFFFFF, 0xFFFFFFFF)])
def test_philox_bit_exact(ctx, c1, c2, c3):
    n = 1 << 18
    for seed in (0, 0x0123456789ABCDEF):
        gpu = ctx.philox_words(seed, 7, c1, c2, c3, n).cpu().numpy().view(np.uint32)
        ref = oracle.philox_words(seed, c1, c2, c3, 7, n)
        assert np.array_equal(gpu, ref)


@pytest.mark.parametrize("sampler", [0, 1, 2])
@pytest.mark.parametrize("D", [1, 2, 3, 9, 64])
@pytest.mark.parametrize("antithetic", [1, 0])
def test_perturbations_match_oracle(ctx, sampler, D, antithetic):
    rng = np.random.default_rng(D)
    sigma = rng.uniform(0.05, 0.5, size=D).astype(np.float32)
    P, seed, step = 16, 1234, 7
    tau, w = ctx.sample_perturbations(_t(sigma), P, sampler=sampler, antithetic=antithetic, seed=seed, step=step)
    tau, w = tau.cpu().numpy(), w.cpu().numpy()
    for r in range(2 * P):
        idx = r // 2 if antithetic else r
        _, tf, wd = oracle.sample(sampler, sigma, seed, step, idx)
        sgn = -1.0 if (antithetic and r % 2) else 1.0
        ref_tau, ref_w = sgn * tf.astype(np.float64), sgn * wd
        scale = np.abs(ref_tau).max()
        assert np.allclose(tau[r], ref_tau, rtol=4e-6, atol=4e-6 * scale), (r, tau[r], ref_tau)
        assert np.allclose(w[r], ref_w, rtol=4e-6, atol=4e-6 * np.abs(ref_w).max()), (r, w[r], ref_w)
        if sampler != 2:
            assert np.array_equal(np.sign(tau[r]), np.sign(ref_tau))


# ---------------------------------------------------------------- images
CASES = {
    "small": lambda: workloads.scaled(workloads.config_small(), width=64, height=64, spp=4),
    "occlusion": lambda: workloads.scaled(workloads.config_occlusion(), width=72, height=52, spp=8),
    "gi-box": lambda: workloads.scaled(workloads.config_gi_box(), width=56, height=40, spp=8),
    "caustic": lambda: workloads.scaled(workloads.config_caustic(), width=48, height=40, spp=16),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("k", [32, 8])
def test_render_matches_oracle(ctx, name, k):
    wl = CASES[name]()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    thetas = np.stack([wl.theta_ref, wl.theta0, wl.theta0 + 0.03]).astype(np.float32)
    img = scene.render_batch(_t(thetas), wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, seed=wl.seed, step=3,
                             tag=2, crn=0, block_pixels=k)
    torch.cuda.synchronize()
    img = img.cpu().numpy()
    ref = oracle.render(wl.scene, wl.bindings, thetas, wl.width, wl.height, wl.spp, wl.depth, wl.rr_start,
                        wl.seed, 3, 2, 0)
    assert np.all(img[..., 3] == 0.0)
    assert_image_parity(img[..., :3], ref, what=f"{name} k={k}")


def test_render_edge_sizes(ctx):
    wl = workloads.config_occlusion()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    for (W, H, spp) in [(1, 1, 1), (7, 3, 2), (17, 33, 1), (33, 17, 3), (5, 9, 40)]:
        for k in (8, 16, 32):
            img = scene.render_batch(_t(wl.theta_ref[None]), W, H, spp, wl.depth, wl.rr_start, seed=1, step=0,
                                     tag=3, crn=1, block_pixels=k).cpu().numpy()
            ref = oracle.render(wl.scene, wl.bindings, wl.theta_ref[None], W, H, spp, wl.depth, wl.rr_start, 1, 0, 3,
                                1)
            diff = np.abs(img[..., :3] - ref)
            assert diff.mean() <= 1e-4 and (diff.max(-1) > 1e-3).sum() <= max(1, int(1e-3 * W * H)), (W, H, k)


# ---------------------------------------------------------------- gradient
def _grad_case(ctx, wl, step=0, k=0):
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = oracle.render_target(wl)
    opts = scene.grad_opts(wl, step=step, block_pixels=k)
    g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), opts)
    torch.cuda.synchronize()
    ref = oracle.smoothed_grad(wl, target=target, step=step)
    return g.cpu().numpy(), L.cpu().numpy(), ref


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_matches_oracle(ctx, name):
    wl = CASES[name]()
    wl.pairs = min(wl.pairs, 8)
    g, L, ref = _grad_case(ctx, wl, step=2)
    assert np.allclose(L, ref["losses"], rtol=1e-4, atol=1e-9), (L, ref["losses"])
    err = grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"])
    assert err <= GRAD_REL, (name, err, g, ref["grad"])


@pytest.mark.parametrize("sampler,antithetic,crn", [(1, 1, 1), (2, 1, 1), (0, 0, 1), (0, 1, 0)])
def test_gradient_estimator_variants(ctx, sampler, antithetic, crn):
    wl = CASES["small"]()
    wl.sampler, wl.antithetic, wl.crn = sampler, antithetic, crn
    g, L, ref = _grad_case(ctx, wl, step=1)
    assert np.allclose(L, ref["losses"], rtol=1e-4, atol=1e-9)
    assert grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL


def test_gradient_full_size_small_config(ctx):
    wl = workloads.config_small()
    for k in (8, 16, 32):
        g, L, ref = _grad_case(ctx, wl, step=0, k=k)
        assert grad_rel_error(g, ref["grad"], ref["weights"], ref["losses"]) <= GRAD_REL, k


def test_invisible_parameter_exact_zero_on_gpu(ctx):
    wl = workloads.scaled(workloads.config_small(), width=32, height=32, spp=2, pairs=4)
    sc = wl.scene
    sc.prim_geom = np.vstack([sc.prim_geom, [[50.0, 50.0, 50.0, 0.05, 0, 0, 0, 0, 0]]]).astype(np.float32)
    sc.prim_type = np.append(sc.prim_type, 0).astype(np.int32)
    sc.prim_mat = np.append(sc.prim_mat, 0).astype(np.int32)
    wl.bindings = np.array([[workloads.BIND_PRIM_POS, sc.n_prims - 1, 0]], np.int32)
    wl.theta0 = wl.theta_ref = np.array([50.0], np.float32)
    wl.sigma = np.array([0.1], np.float32)
    g, L, _ = _grad_case(ctx, wl)
    assert g[0] == 0.0 and np.array_equal(L[0::2], L[1::2])


def test_deterministic_across_launch_shapes(ctx):
    wl = CASES["occlusion"]()
    wl.pairs = 4
    g1, L1, _ = _grad_case(ctx, wl, k=32)
    g1b, L1b, _ = _grad_case(ctx, wl, k=32)
    assert np.array_equal(g1, g1b) and np.array_equal(L1, L1b)  # bitwise reproducible
    g4, L4, ref = _grad_case(ctx, wl, k=8)
    assert np.allclose(L4, L1, rtol=1e-12)  # block shape changes only the FP64 summation grouping


def _occlusion_with_albedo():
    """The box's position and a sphere's red albedo: a path that meets the sphere is traced
    again by every render from that vertex on, one that touched the box's bounds before
    from its first touch."""
    wl = workloads.scaled(workloads.config_occlusion(), width=48, height=40, spp=4, pairs=4)
    sph = int(wl.scene.prim_mat[1])
    wl.bindings = np.vstack([wl.bindings, [[workloads.BIND_MAT_ALBEDO, sph, 0]]]).astype(np.int32)
    wl.theta_ref = np.append(wl.theta_ref, 0.6).astype(np.float32)
    wl.theta0 = np.append(wl.theta0, 0.85).astype(np.float32)
    wl.sigma = np.append(wl.sigma, 0.05).astype(np.float32)
    return wl


def _moving_primitive(wl, prim, offset):
    """wl with theta = the position of primitive `prim` (sigma 0.05), started at `offset`."""
    c0 = wl.scene.prim_geom[prim, :3].astype(np.float32)
    wl.bindings = np.array([[workloads.BIND_PRIM_POS, prim, c] for c in range(3)], np.int32)
    wl.theta_ref = c0.copy()
    wl.theta0 = (c0 + np.asarray(offset, np.float32)).astype(np.float32)
    wl.sigma = np.full(3, 0.05, np.float32)
    return wl


def _gi_box_moving_box():
    """The GI box with a moving box beside the mirror sphere (mirror bounces, Russian
    roulette): renders resume after specular vertices with their emission flag."""
    wl = workloads.scaled(workloads.config_gi_box(), width=40, height=32, spp=4, pairs=3)
    return _moving_primitive(wl, 5, (0.05, -0.03, 0.0))


def _caustic_moving_glass():
    """The caustic scene with the glass sphere moving: paths refract through the moving
    primitive and reach the light after dielectric bounces."""
    wl = workloads.scaled(workloads.config_caustic(), width=40, height=40, spp=4, pairs=3)
    return _moving_primitive(wl, 1, (0.04, 0.02, -0.03))


def _small_pool_overflow():
    """sigma = 1.5: the union of the sphere's bounds covers the view, every path touches it
    and the segment pool (4096 paths here) runs out; the later paths are traced again from
    the camera."""
    wl = workloads.scaled(workloads.config_small(), pairs=4)
    wl.sigma = np.full_like(wl.sigma, 1.5)
    return wl


@pytest.mark.parametrize("make", [workloads.config_small, workloads.config_occlusion,
                                  lambda: workloads.scaled(workloads.config_occlusion(), width=45, height=37, spp=7),
                                  # 64 renders: the render mask uses all 64 bits
                                  lambda: workloads.scaled(workloads.config_occlusion(), width=64, height=48, spp=4,
                                                           pairs=32),
                                  # 80 renders: a touched path is traced again by every render
                                  lambda: workloads.scaled(workloads.config_occlusion(), width=40, height=40, spp=4,
                                                           pairs=40),
                                  # depth 6 with Russian roulette: renders resume mid-path
                                  lambda: workloads.scaled(workloads.config_occlusion(), width=48, height=40, spp=4,
                                                           pairs=4, depth=6, rr_start=2),
                                  _occlusion_with_albedo, _small_pool_overflow, _gi_box_moving_box,
                                  _caustic_moving_glass])
def test_path_sharing_is_bit_identical(ctx, make):
    """With common random numbers, a path is traced once in the scene without the
    perturbed primitives; only the renders whose own primitives one of its rays may meet
    trace it again, and add their radiance minus the shared one. The gradient and losses
    must equal tracing every path in every render."""
    wl = make()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = _t(oracle.render_target(wl))
    res = []
    for no_share in (0, 1):
        opts = scene.grad_opts(wl, step=5, no_path_sharing=no_share)
        g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), target, opts)
        torch.cuda.synchronize()
        res.append((g.cpu().numpy(), L.cpu().numpy()))
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][0], res[1][0])
    # and sharing was in use: fewer paths traced than every render tracing every path
    ctx.counters_enable(True)
    scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), target, scene.grad_opts(wl, step=5))
    paths = ctx.counters_read()[3]
    ctx.counters_enable(False)
    assert 0 < paths < wl.renders * wl.width * wl.height * wl.spp


def _grad_and_paths(ctx, scene, wl, target, opts, paths, key):
    """The gradient and losses of the timed kernels, and (in a second, counted call) the
    paths they trace. The counting variants are separate code and are compared with the
    timed kernels only through their counts."""
    g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), target, opts)
    torch.cuda.synchronize()
    ctx.counters_enable(True)
    scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), target, opts)
    torch.cuda.synchronize()
    paths[key] = ctx.counters_read()[3]
    ctx.counters_enable(False)
    return g.cpu().numpy(), L.cpu().numpy()


def _small_radius_bound():
    """The small scene with the sphere's radius bound beside its position (an emitter-free
    radius binding: per-render areas rows in render-group mode)."""
    wl = workloads.scaled(workloads.config_small(), width=40, height=36, spp=4, pairs=4)
    wl.bindings = np.concatenate([wl.bindings, np.array([[workloads.BIND_SPHERE_RADIUS, 1, 0]], np.int32)])
    wl.theta0 = np.concatenate([wl.theta0, [0.5]]).astype(np.float32)
    wl.theta_ref = np.concatenate([wl.theta_ref, [0.45]]).astype(np.float32)
    wl.sigma = np.concatenate([wl.sigma, [0.05]]).astype(np.float32)
    return wl


@pytest.mark.parametrize("make,groups", [
    # the caustic task: 64 renders, the light moves (a perturbed emitter in every lane's records)
    (lambda: workloads.scaled(workloads.config_caustic(), width=72, height=52, spp=4, pairs=32), (0, 32, 8, 2)),
    # the GI box: the light moves and two walls' albedos are bound (per-render materials)
    (lambda: workloads.scaled(workloads.config_gi_box(), width=48, height=40, spp=4, pairs=16), (0, 32, 16, 4)),
    # a bound radius (emitter areas per render) on the small scene's sphere
    (_small_radius_bound, (0, 8)),
    # ragged blocks, renders not a multiple of 4
    (lambda: workloads.scaled(workloads.config_caustic(), width=37, height=29, spp=3, pairs=3), (0, 2)),
    # a moving box with path sharing off, and Russian roulette
    (lambda: workloads.scaled(workloads.config_occlusion(), width=48, height=40, spp=4, pairs=4, depth=6,
                              rr_start=2), (0, 8, 2)),
])
@pytest.mark.parametrize("block_pixels", [8, 32])
def test_render_groups_are_bit_identical(ctx, make, groups, block_pixels):
    """Render-group mode traces each path sample for several renders side by side (one lane
    per render) with the invariant scene shared and each lane's perturbed primitives and
    materials its own: every loss and the gradient equal tracing one render per work item,
    bit for bit, for every group size, and the same paths are traced."""
    wl = make()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = _t(oracle.render_target(wl))
    res, paths = {}, {}
    for rg in (-1,) + tuple(groups):
        opts = scene.grad_opts(wl, step=3, block_pixels=block_pixels, no_path_sharing=1, render_groups=rg)
        res[rg] = _grad_and_paths(ctx, scene, wl, target, opts, paths, rg)
    for rg in groups:
        assert np.array_equal(res[rg][1], res[-1][1]), (rg, res[rg][1], res[-1][1])
        assert np.array_equal(res[rg][0], res[-1][0]), (rg, res[rg][0], res[-1][0])
        assert paths[rg] == paths[-1] == wl.renders * wl.width * wl.height * wl.spp


def test_render_groups_match_oracle(ctx):
    """The caustic and GI-box gradients in render-group mode against the FP64 oracle."""
    for wl in (workloads.scaled(workloads.config_caustic(), width=64, height=48, spp=4, pairs=8),
               workloads.scaled(workloads.config_gi_box(), width=48, height=40, spp=4, pairs=8)):
        scene = ctx.upload_scene(wl.scene, wl.bindings)
        target = oracle.render_target(wl)
        opts = scene.grad_opts(wl, step=1, render_groups=16, no_path_sharing=1)
        g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), opts)
        torch.cuda.synchronize()
        ref = oracle.smoothed_grad(wl, target=target, step=1)
        err = grad_rel_error(g.cpu().numpy(), ref["grad"], ref["weights"], ref["losses"])
        assert err <= GRAD_REL, (wl.name, err)


def _gi_box_moving_light():
    """The GI box with only its light moving: long diffuse paths (more kept vertices than
    the emitter-sharing mode keeps), mirror bounces and Russian roulette."""
    wl = workloads.scaled(workloads.config_gi_box(), width=40, height=32, spp=5, pairs=3)
    return _moving_primitive(wl, 8, (0.05, -0.03, -0.02))


def _caustic_two_lights():
    """The caustic scene with a second emitter, a small sphere whose radius is bound beside
    the quad light's position: the next-event estimate first chooses an emitter, and the
    sphere's area differs between renders."""
    wl = workloads.scaled(workloads.config_caustic(), width=40, height=36, spp=4, pairs=4)
    b = workloads.SceneBuilder()
    m_floor = b.material(workloads.MAT_DIFFUSE, (0.8, 0.8, 0.8))
    m_glass = b.material(workloads.MAT_DIELECTRIC, (1.0, 1.0, 1.0), ior=1.5)
    m_light = b.material(workloads.MAT_DIFFUSE, (0.0, 0.0, 0.0), emission=(200.0, 200.0, 200.0))
    m_bulb = b.material(workloads.MAT_DIFFUSE, (0.0, 0.0, 0.0), emission=(30.0, 20.0, 10.0))
    b.quad((0, 0, 0), (10, 0, 0), (0, 10, 0), m_floor)
    b.sphere((0.0, 0.0, 1.0), 0.5, m_glass)
    bulb = b.sphere((-0.8, 0.6, 2.0), 0.15, m_bulb)
    light = b.quad((0.6, 0.4, 2.6), (0.2, 0, 0), (0, -0.2, 0), m_light)
    b.look_at((0, -4.0, 1.2), (0, 0, 0.6), (0, 0, 1), 40.0)
    wl.scene = b.build()
    wl.bindings = np.array([[workloads.BIND_PRIM_POS, light, c] for c in range(3)]
                           + [[workloads.BIND_SPHERE_RADIUS, bulb, 0]], np.int32)
    wl.theta_ref = np.array([0.6, 0.4, 2.6, 0.15], np.float32)
    wl.theta0 = np.array([0.5, 0.3, 2.5, 0.2], np.float32)
    wl.sigma = np.array([0.125, 0.125, 0.125, 0.03], np.float32)
    return wl


@pytest.mark.parametrize("make,block_pixels", [
    # the caustic task's 64 renders
    (lambda: workloads.scaled(workloads.config_caustic(), width=72, height=52, spp=4, pairs=32), 8),
    (lambda: workloads.scaled(workloads.config_caustic(), width=72, height=52, spp=4, pairs=32), 32),
    # ragged blocks, 6 renders
    (lambda: workloads.scaled(workloads.config_caustic(), width=37, height=29, spp=3, pairs=3), 8),
    # 40 samples (a second, partial round of 32) and 48 renders (a lane's second render
    # only for lanes 0-15)
    (lambda: workloads.scaled(workloads.config_caustic(), width=24, height=20, spp=40, pairs=24), 16),
    # no Russian roulette, depth 3: the last vertex's estimate and the depth limit
    (lambda: workloads.scaled(workloads.config_caustic(), width=40, height=32, spp=4, pairs=4, depth=3,
                              rr_start=-1), 8),
    (_gi_box_moving_light, 8),
    (_gi_box_moving_light, 32),
    (_caustic_two_lights, 16),
])
def test_emitter_sharing_is_bit_identical(ctx, make, block_pixels):
    """Emitter sharing traces each path once in the invariant scene, keeps its diffuse
    vertices, and lets every render add its own next-event estimates there (and trace on
    where a ray could meet its perturbed primitives): every loss and the gradient equal
    tracing one render per work item, and render groups, bit for bit."""
    wl = make()
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = _t(oracle.render_target(wl))
    res, paths = {}, {}
    for key, kw in (("emit", {}), ("per-render", dict(no_path_sharing=1, render_groups=-1)),
                    ("groups", dict(no_path_sharing=1))):
        opts = scene.grad_opts(wl, step=4, block_pixels=block_pixels, **kw)
        res[key] = _grad_and_paths(ctx, scene, wl, target, opts, paths, key)
    for key in ("per-render", "groups"):
        assert np.array_equal(res["emit"][1], res[key][1]), (key, res["emit"][1], res[key][1])
        assert np.array_equal(res["emit"][0], res[key][0]), (key, res["emit"][0], res[key][0])
    # each path sample was traced once for all renders
    assert paths["emit"] == wl.width * wl.height * wl.spp < paths["per-render"]


def test_emitter_sharing_falls_back_beyond_64_renders(ctx):
    """A moving-light job with more renders than emitter sharing serves (80) runs in render
    groups: every path of every render is traced, with the same results as path sharing off."""
    wl = workloads.scaled(workloads.config_caustic(), width=24, height=20, spp=2, pairs=40)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = _t(oracle.render_target(wl))
    res, paths = [], {}
    for no_share in (0, 1):
        opts = scene.grad_opts(wl, step=2, block_pixels=8, no_path_sharing=no_share)
        res.append(_grad_and_paths(ctx, scene, wl, target, opts, paths, no_share))
        assert paths[no_share] == wl.renders * wl.width * wl.height * wl.spp
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_emitter_sharing_matches_oracle(ctx):
    """The caustic and moving-light GI-box gradients in emitter-sharing mode against the
    FP64 oracle."""
    for wl in (workloads.scaled(workloads.config_caustic(), width=64, height=48, spp=4, pairs=8),
               _gi_box_moving_light(), _caustic_two_lights()):
        scene = ctx.upload_scene(wl.scene, wl.bindings)
        target = oracle.render_target(wl)
        opts = scene.grad_opts(wl, step=1)
        ctx.counters_enable(True)
        g, L = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target), opts)
        torch.cuda.synchronize()
        paths = ctx.counters_read()[3]
        ctx.counters_enable(False)
        assert paths == wl.width * wl.height * wl.spp  # the mode was in use
        ref = oracle.smoothed_grad(wl, target=target, step=1)
        err = grad_rel_error(g.cpu().numpy(), ref["grad"], ref["weights"], ref["losses"])
        assert err <= GRAD_REL, (wl.name, err)


def test_host_buffer_gradient_equals_device_call(ctx):
    """prdpt_smoothed_grad_host (inputs and results in host memory, pageable or
    page-locked, on the default or another stream) returns the device call's gradient and
    losses bit for bit, call after call with changing targets."""
    wl = workloads.scaled(workloads.config_occlusion(), width=48, height=40, spp=4, pairs=4)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = oracle.render_target(wl).astype(np.float32)
    opts = scene.grad_opts(wl, step=3)
    side = torch.cuda.Stream()
    # the target travels on a stream of its own: alternate two targets so that a result
    # computed before its target arrived would show
    for target_k in (target, 0.5 * target, target):
        g_dev, L_dev = scene.smoothed_grad(_t(wl.theta0), _t(wl.sigma), _t(target_k), opts)
        torch.cuda.synchronize()
        for pinned in (False, True):
            th, sg, tg = (np.ascontiguousarray(a, np.float32) for a in (wl.theta0, wl.sigma, target_k))
            if pinned:
                th, sg, tg = (torch.from_numpy(a).pin_memory() for a in (th, sg, tg))
            for stream in (None, side):
                g, L = scene.smoothed_grad_host(th, sg, tg, opts, stream=stream)
                assert np.array_equal(g, g_dev.cpu().numpy()) and np.array_equal(L, L_dev.cpu().numpy())


def _host_step_case(name):
    if name == "occlusion":  # Eq. 10 with path sharing: Adam in k_finalize
        return workloads.scaled(workloads.config_occlusion(), width=40, height=32, spp=4, pairs=3)
    if name == "albedo":  # Eq. 9: Adam after the mean of the pathwise render gradients
        return workloads.scaled(workloads.config_small_albedo(), width=24, height=16, spp=4, pairs=2)
    wl = workloads.config_texture(res=8, px_per_texel=2)  # D = 192: Adam in k_hd_grad
    wl.pairs, wl.spp = 3, 2
    return wl


@pytest.mark.parametrize("name", ["occlusion", "albedo", "texture"])
def test_host_buffer_step_follows_the_device_calls(ctx, name):
    """prdpt_step_host (gradient and Adam with theta, m, v in host memory; the update taken
    by the gradient's last kernel) follows, bit for bit over three steps, the trajectory of
    prdpt_smoothed_grad plus prdpt_adam_step on device buffers, and a gradient-only host
    call between its steps leaves it unchanged."""
    wl = _host_step_case(name)
    scene = ctx.upload_scene(wl.scene, wl.bindings)
    target = oracle.render_target(wl).astype(np.float32)
    th_d, m_d, v_d = _t(wl.theta0), torch.zeros(wl.D, device="cuda"), torch.zeros(wl.D, device="cuda")
    th_h = np.ascontiguousarray(wl.theta0, np.float32)
    m_h, v_h = np.zeros(wl.D, np.float32), np.zeros(wl.D, np.float32)
    g_h, L_h = np.empty(wl.D, np.float32), np.empty(wl.renders, np.float32)
    sg, tg = np.ascontiguousarray(wl.sigma, np.float32), np.ascontiguousarray(target)
    for t in range(3):
        opts = scene.grad_opts(wl, step=t)
        g_d, L_d = scene.smoothed_grad(th_d, _t(wl.sigma), _t(target), opts)
        ctx.adam_step(th_d, m_d, v_d, g_d, t + 1, wl.lr)
        scene.step_host(th_h, m_h, v_h, t + 1, wl.lr, sg, tg, opts, grad=g_h, losses=L_h)
        torch.cuda.synchronize()
        assert np.array_equal(g_h, g_d.cpu().numpy()) and np.array_equal(L_h, L_d.cpu().numpy())
        for host, dev in ((th_h, th_d), (m_h, m_d), (v_h, v_d)):
            assert np.array_equal(host, dev.cpu().numpy())
        g2, L2 = scene.smoothed_grad_host(th_h, sg, tg, opts)
        g2_d, L2_d = scene.smoothed_grad(th_d, _t(wl.sigma), _t(target), opts)
        assert np.array_equal(g2, g2_d.cpu().numpy()) and np.array_equal(L2, L2_d.cpu().numpy())
