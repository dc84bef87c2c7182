"""Pins of the oracle's forward model P(theta) (Eq. 1, Eq. 3) by physics and geometry.

* White furnace: a convex diffuse (or mirror) object of albedo rho under a
  uniform environment of radiance 1 shows exactly rho; with rho = 1 the object
  vanishes.
* Analytic irradiance: a uniform spherical emitter (radius r, radiance Le) fully
  above a surface point gives E = pi Le r^2 cos(beta) / d^2; a uniform polygonal
  emitter gives Lambert's closed form E = Le/2 sum_i angle_i (n . unit(v_i x v_i+1)).
  A diffuse surface of albedo rho then shows rho E / pi, averaged over the pixel
  footprint.
* Geometry and visibility: an emitting rectangle aligned with the pixel grid is
  seen in exactly the pixels it covers, so the loss between two positions is the
  symmetric-difference area (the circle example of Fig. 2, with rectangles), and
  it is flat (a plateau) once the two do not overlap.
* Ray-primitive hits against hand-computed values.
"""
import math

import numpy as np
import pytest

import oracle
from workloads import (BIND_MAT_ALBEDO, BIND_PRIM_POS, MAT_DIELECTRIC, MAT_DIFFUSE, MAT_MIRROR,
                       SceneBuilder)


def _render(scene, W, H, spp, depth, theta=None, binds=None, seed=1, crn=1):
    if binds is None:
        binds = np.zeros((1, 3), np.int32)  # a harmless binding: albedo R of material 0 set to its own value
        binds[0] = [BIND_MAT_ALBEDO, 0, 0]
        theta = np.array([[scene.mat_param[0, 0]]], np.float32)
    return oracle.render(scene, binds, np.atleast_2d(theta), W, H, spp, depth, -1, seed, 0, oracle.TAG_PATH, crn)


# ---------------------------------------------------------------- furnace
@pytest.mark.parametrize("kind,rho", [(MAT_DIFFUSE, 0.6), (MAT_DIFFUSE, 1.0), (MAT_MIRROR, 0.35)])
def test_white_furnace(kind, rho):
    b = SceneBuilder()
    m = b.material(kind, (rho, rho, rho))
    b.sphere((0, 0, 0), 1.0, m)
    b.look_at((0, -5, 0), (0, 0, 0), (0, 0, 1), 40.0)
    b.background[:] = 1.0
    sc = b.build()
    W = H = 32
    S = 8
    img = _render(sc, W, H, S, depth=3)[0]
    rho = float(np.float32(rho))  # the scene stores FP32 values
    # each sample sees either the environment (1) or the object once (rho): pixel = 1 - k(1 - rho)/S
    if rho == 1.0:
        assert np.all(np.abs(img - 1.0) < 1e-14)
        return
    k = (1.0 - img) * S / (1.0 - rho)
    assert np.all(np.abs(k - np.round(k)) < 1e-9) and np.all((k > -1e-9) & (k < S + 1e-9))
    assert np.allclose(img[H // 2, W // 2], rho, atol=1e-14)
    assert np.allclose(img[0, 0], 1.0, atol=1e-14)
    assert np.allclose(img[..., 0], img[..., 1]) and np.allclose(img[..., 0], img[..., 2])


def test_dielectric_furnace_conserves_energy():
    b = SceneBuilder()
    m = b.material(MAT_DIELECTRIC, (1, 1, 1), ior=1.5)
    b.sphere((0, 0, 0), 1.0, m)
    b.look_at((0, -5, 0), (0, 0, 0), (0, 0, 1), 40.0)
    b.background[:] = 1.0
    img = _render(b.build(), 16, 16, 16, depth=64)[0]
    # no absorption: every path that escapes carries exactly 1; only paths cut at the
    # depth limit carry 0
    assert np.all(img <= 1.0 + 1e-12) and img.mean() > 0.995


# ---------------------------------------------------------------- irradiance
def _camera_rays(cam, W, H, jit):
    eye, look, up, fov = cam[0:3].astype(np.float64), cam[3:6].astype(np.float64), cam[6:9].astype(np.float64), float(cam[9])
    f = look - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(fov) / 2)
    g = (np.arange(jit) + 0.5) / jit
    xs = (np.arange(W)[:, None] + g[None, :]).reshape(-1)
    ys = (np.arange(H)[:, None] + g[None, :]).reshape(-1)
    sx = (2 * xs / W - 1) * (W / H) * th
    sy = (1 - 2 * ys / H) * th
    d = f[None, None] + sy[:, None, None] * u[None, None] + sx[None, :, None] * r[None, None]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return eye, d  # d: [H*jit, W*jit, 3]


def _plane_points(eye, d):
    t = -eye[2] / d[..., 2]
    return eye[None, None] + t[..., None] * d


def _footprint_average(field, W, H, jit):
    return field.reshape(H, jit, W, jit).mean(axis=(1, 3))


def _ground_scene(light_kind):
    b = SceneBuilder()
    m_ground = b.material(MAT_DIFFUSE, (0.5, 0.5, 0.5))
    b.quad((0, 0, 0), (20, 0, 0), (0, 20, 0), m_ground)
    if light_kind == "sphere":
        m_l = b.material(MAT_DIFFUSE, (0, 0, 0), emission=(20, 20, 20))
        b.sphere((1.5, 0.0, 1.0), 0.2, m_l)
    else:
        m_l = b.material(MAT_DIFFUSE, (0, 0, 0), emission=(10, 10, 10))
        b.quad((1.2, 0.0, 1.5), (0.5, 0, 0), (0, -0.5, 0), m_l)
    b.look_at((0, 0, 4), (0, 0, 0), (0, 1, 0), 20.0)
    return b.build()


def _lambert_polygon_irradiance(points, verts, Le):
    """E at points (normal +z) from a uniform polygon of radiance Le (Lambert's formula)."""
    E = np.zeros(points.shape[:-1])
    n = len(verts)
    for i in range(n):
        a = verts[i][None, None] - points
        b = verts[(i + 1) % n][None, None] - points
        an = a / np.linalg.norm(a, axis=-1, keepdims=True)
        bn = b / np.linalg.norm(b, axis=-1, keepdims=True)
        ang = np.arccos(np.clip((an * bn).sum(-1), -1, 1))
        c = np.cross(a, b)
        c /= np.linalg.norm(c, axis=-1, keepdims=True)
        E += ang * c[..., 2]
    return np.abs(E) * Le / 2


@pytest.mark.parametrize("light_kind", ["sphere", "quad"])
def test_direct_lighting_matches_closed_form(light_kind):
    sc = _ground_scene(light_kind)
    W = H = 32
    S = 1024
    img = _render(sc, W, H, S, depth=1, seed=7)[0][..., 0]
    jit = 6
    eye, d = _camera_rays(sc.camera, W, H, jit)
    pts = _plane_points(eye, d)
    rho = 0.5
    if light_kind == "sphere":
        c = np.array([1.5, 0.0, 1.0])
        r, Le = 0.2, 20.0
        v = c[None, None] - pts
        dist = np.linalg.norm(v, axis=-1)
        E = math.pi * Le * r * r * (v[..., 2] / dist) / dist ** 2
    else:
        c, hu, hv = np.array([1.2, 0.0, 1.5]), np.array([0.25, 0, 0]), np.array([0, 0.25, 0])
        verts = [c - hu - hv, c + hu - hv, c + hu + hv, c - hu + hv]
        E = _lambert_polygon_irradiance(pts, verts, 10.0)
    expect = _footprint_average(rho * E / math.pi, W, H, jit)
    assert img.mean() == pytest.approx(expect.mean(), rel=1e-2)
    blocks = lambda a: a.reshape(4, 8, 4, 8).mean(axis=(1, 3))  # noqa: E731
    assert np.allclose(blocks(img), blocks(expect), rtol=2.5e-2)


# ---------------------------------------------------------------- geometry / visibility
def _rect_scene():
    """Camera at height 5 looking down; an emitting rectangle (radiance 1, facing up)
    at height 1 whose centre is bound to theta (x, y). tan(fov/2) = 1/2 makes the
    pixel footprint at distance 4 exactly 1/16, so pixel-aligned positions are
    exact in FP32."""
    b = SceneBuilder()
    m = b.material(MAT_DIFFUSE, (0, 0, 0), emission=(1, 1, 1))
    W = 64
    px = 2 * 4.0 * 0.5 / W  # = 1/16
    rect = b.quad((0, 0, 1), (10 * px, 0, 0), (0, 6 * px, 0), m)
    b.look_at((0, 0, 5), (0, 0, 0), (0, 1, 0), math.degrees(2 * math.atan(0.5)))
    binds = np.array([[BIND_PRIM_POS, rect, 0], [BIND_PRIM_POS, rect, 1]], np.int32)
    return b.build(), binds, px, W


def _rect_mask(cx_px, cy_px, W):
    """Pixels covered by a 10x6-pixel rectangle centred at pixel offset (cx, cy) from the image centre."""
    m = np.zeros((W, W), bool)
    x0 = W // 2 + cx_px - 5
    y0 = W // 2 - cy_px - 3  # image y runs down, scene y runs up
    m[y0:y0 + 6, x0:x0 + 10] = True
    return m


def test_pixel_aligned_rectangle_is_seen_exactly():
    sc, binds, px, W = _rect_scene()
    positions = [(0, 0), (7, -4), (-12, 9)]
    thetas = np.array([[cx * px, cy * px] for cx, cy in positions], np.float32)
    imgs = oracle.render(sc, binds, thetas, W, W, 16, 1, -1, 3, 0, oracle.TAG_PATH, 1)
    for img, (cx, cy) in zip(imgs, positions):
        assert np.array_equal(img[..., 0] == 1.0, _rect_mask(cx, cy, W))
        assert set(np.unique(img)) <= {0.0, 1.0}


def test_loss_is_symmetric_difference_and_plateau():
    sc, binds, px, W = _rect_scene()
    ref = (0, 0)
    target = np.zeros((W, W, 4), np.float32)
    target[..., :3] = _rect_mask(*ref, W)[..., None]
    for cx, cy in [(0, 0), (3, 0), (4, 2), (9, 5), (14, 0), (20, -12)]:
        img = oracle.render(sc, binds, np.array([[cx * px, cy * px]], np.float32), W, W, 8, 1, -1, 3, 0,
                            oracle.TAG_PATH, 1)[0]
        sym = np.logical_xor(_rect_mask(cx, cy, W), _rect_mask(*ref, W)).sum()
        assert oracle.mse(img, target) == pytest.approx(sym / (W * W), rel=1e-12, abs=1e-15)
    # far from the reference the unsmoothed loss is flat (a plateau) ...
    far = [oracle.mse(oracle.render(sc, binds, np.array([[cx * px, 0]], np.float32), W, W, 8, 1, -1, 3, 0,
                                    oracle.TAG_PATH, 1)[0], target) for cx in (14, 15, 18)]
    assert far[0] == far[1] == far[2]


def test_smoothed_gradient_leaves_the_plateau_towards_the_reference():
    """Fig. 2: from a non-overlapping start the plain gradient is zero, while the
    plateau-reduced gradient points towards the reference."""
    sc, binds, px, W = _rect_scene()
    from workloads import Workload
    target = np.zeros((W, W, 4), np.float32)
    target[..., :3] = _rect_mask(0, 0, W)[..., None]
    wl = Workload(name="rect", scene=sc, bindings=binds, theta_ref=np.zeros(2, np.float32),
                  theta0=np.array([12 * px, 7 * px], np.float32), sigma=np.array([0.4, 0.4], np.float32),
                  width=W, height=W, spp=4, depth=1, rr_start=-1, pairs=64, seed=2)
    g = oracle.smoothed_grad(wl, target=target)["grad"]
    descent = -g
    to_ref = -wl.theta0.astype(np.float64)
    cos = descent @ to_ref / (np.linalg.norm(descent) * np.linalg.norm(to_ref))
    assert cos > 0.8
    h = 1e-3
    Lp = oracle.mse(oracle.render(sc, binds, (wl.theta0 + [h, 0])[None], W, W, 4, 1, -1, 2, 0, oracle.TAG_PATH, 1)[0], target)
    Lm = oracle.mse(oracle.render(sc, binds, (wl.theta0 - [h, 0])[None], W, W, 4, 1, -1, 2, 0, oracle.TAG_PATH, 1)[0], target)
    assert Lp == Lm  # zero plain gradient on the plateau


def _prim_scene():
    b = SceneBuilder()
    m = b.material()
    b.sphere((0, 0, 0), 1.0, m)                      # 0
    b.quad((0, 0, 2), (2, 0, 0), (0, 1, 0), m)       # 1: 2 x 1 in the plane z = 2, normal +z
    b.box((5, 0, 0), (1, 0.5, 0.25), m)              # 2
    return b.build()


@pytest.mark.parametrize("prim,o,d,t,n", [
    (0, (0, 0, -5), (0, 0, 1), 4.0, (0, 0, -1)),
    (0, (0, 0, 0), (1, 0, 0), 1.0, (1, 0, 0)),                      # from inside: the far hit
    (0, (0, 0.6, -5), (0, 0, 1), 5 - math.sqrt(1 - 0.36), (0, 0.6, -math.sqrt(0.64))),
    (0, (0, 1.01, -5), (0, 0, 1), math.inf, None),                   # passes beside
    (0, (0, 0, 5), (0, 0, 1), math.inf, None),                       # behind the origin
    (1, (0.5, 0.25, 0), (0, 0, 1), 2.0, (0, 0, 1)),
    (1, (0.5, 0.25, 4), (0, 0, -1), 2.0, (0, 0, 1)),                 # geometric normal, either side
    (1, (1.1, 0, 0), (0, 0, 1), math.inf, None),                     # outside the 2 x 1 extent in x
    (1, (0, 0.6, 0), (0, 0, 1), math.inf, None),                     # outside in y
    (1, (0, 0, 0), (1, 0, 0), math.inf, None),                       # parallel
    (2, (0, 0, 0), (1, 0, 0), 4.0, (-1, 0, 0)),
    (2, (5, 3, 0), (0, -1, 0), 2.5, (0, 1, 0)),
    (2, (5, 0, -3), (0, 0, 1), 2.75, (0, 0, -1)),
    (2, (5, 0, 0), (0, 0, 1), 0.25, (0, 0, 1)),                      # from inside
    (2, (0, 0.6, 0), (1, 0, 0), math.inf, None),
    (2, (0, 0, 0), (-1, 0, 0), math.inf, None),
])
def test_ray_primitive_hits(prim, o, d, t, n):
    tt, nn = oracle.intersect(_prim_scene(), prim, np.array(o, float), np.array(d, float))
    if math.isinf(t):
        assert math.isinf(tt)
    else:
        assert tt == pytest.approx(t, rel=1e-12)
        assert np.allclose(nn, n, atol=1e-12)


def test_one_sided_quad_emitter_and_shadow():
    """A downward-facing light is dark from above and lights the floor; an occluder
    between them casts a shadow whose centre is exactly black at depth 1."""
    b = SceneBuilder()
    m_floor = b.material(MAT_DIFFUSE, (0.5, 0.5, 0.5))
    m_l = b.material(MAT_DIFFUSE, (0, 0, 0), emission=(5, 5, 5))
    m_occ = b.material(MAT_DIFFUSE, (0.5, 0.5, 0.5))
    b.quad((0, 0, 0), (20, 0, 0), (0, 20, 0), m_floor)
    b.quad((0, 0, 2), (0.2, 0, 0), (0, -0.2, 0), m_l)   # normal -z: emits downwards
    b.box((0, 0, 1), (0.3, 0.3, 0.05), m_occ)
    b.look_at((0.9, 0, 5), (0.9, 0, 0), (0, 1, 0), 30.0)
    sc = b.build()
    img = _render(sc, 32, 32, 4, depth=1)[0]
    # the occluder's shadow (below the light) lies around x = 0: left edge of this view
    # is not in shadow; the light seen from above (back side) would be black anyway.
    assert img[16, 31, 0] > 0 and img[16, 31, 0] < 1
    b2 = SceneBuilder()
    m_l2 = b2.material(MAT_DIFFUSE, (0, 0, 0), emission=(5, 5, 5))
    b2.quad((0, 0, 0), (1, 0, 0), (0, 1, 0), m_l2)      # normal +z
    b2.look_at((0, 0, 3), (0, 0, 0), (0, 1, 0), 15.0)
    up = _render(b2.build(), 8, 8, 2, depth=1)[0]
    b3 = SceneBuilder()
    m_l3 = b3.material(MAT_DIFFUSE, (0, 0, 0), emission=(5, 5, 5))
    b3.quad((0, 0, 0), (1, 0, 0), (0, -1, 0), m_l3)     # normal -z: seen from behind
    b3.look_at((0, 0, 3), (0, 0, 0), (0, 1, 0), 15.0)
    down = _render(b3.build(), 8, 8, 2, depth=1)[0]
    assert np.all(up[..., 0] == 5.0) and np.all(down == 0.0)
