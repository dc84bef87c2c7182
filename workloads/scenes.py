"""Synthetic scenes shaped like the paper's optimisation tasks (Sec. 4.1, Supp. Tab. 1).

The paper's own Mitsuba scenes (cup mesh, Cornell box, glass sphere) are not
available, so every workload here is a seeded analytic stand-in with the shape
of one task: image size, number of perturbations N, samples per pixel, path
depth, parameter dimension and kernel bandwidth sigma.

Conventions (shared by both implementations, stated once here):

* z is up, positions are in scene units, colours are linear RGB.
* Primitive geometry is 9 floats per primitive:
    sphere: centre(3), radius, unused(5)
    quad:   centre(3), edge u(3), edge v(3); corners c +- u/2 +- v/2, the
            edges are orthogonal, the normal is normalize(u x v) and a
            one-sided emitter radiates into the half-space the normal points to
    box:    centre(3), half-size(3), unused(3) (axis aligned)
* Materials are 8 floats: albedo(3), emission(3), index of refraction, unused.
* Camera is 10 floats: eye(3), look-at(3), up(3), vertical field of view in
  degrees.
* A parameter binding (kind, index, component) makes theta_d *set* one scene
  field: the position (centre) of primitive `index`, the radius of sphere
  `index`, or the albedo / emission channel of material `index`.
* The number of antithetic pairs P is given explicitly; a workload renders
  R = 2P perturbed scenes per step (the paper's N counts renders, Supp. Sec. 2:
  N=2 is one sample and its antithesis).
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field, replace

import numpy as np

PRIM_SPHERE, PRIM_QUAD, PRIM_BOX = 0, 1, 2
MAT_DIFFUSE, MAT_MIRROR, MAT_DIELECTRIC = 0, 1, 2
BIND_PRIM_POS, BIND_SPHERE_RADIUS, BIND_MAT_ALBEDO, BIND_MAT_EMISSION = 0, 1, 2, 3
BIND_TEXTURE = 4  # one row (4, material, T) standing for the T x T x 3 texel albedos
SAMPLER_RADIAL, SAMPLER_PERDIM, SAMPLER_GAUSS = 0, 1, 2


@dataclass
class Scene:
    prim_type: np.ndarray   # int32 [n]
    prim_mat: np.ndarray    # int32 [n]
    prim_geom: np.ndarray   # float32 [n, 9]
    mat_type: np.ndarray    # int32 [m]
    mat_param: np.ndarray   # float32 [m, 8]
    camera: np.ndarray      # float32 [10]
    background: np.ndarray  # float32 [3]

    @property
    def n_prims(self) -> int:
        return int(self.prim_type.shape[0])

    @property
    def n_mats(self) -> int:
        return int(self.mat_type.shape[0])


class SceneBuilder:
    """Small helper that accumulates primitives and materials into a Scene."""

    def __init__(self):
        self._types, self._mats, self._geom = [], [], []
        self._mtypes, self._mparams = [], []
        self.camera = np.zeros(10, np.float32)
        self.background = np.zeros(3, np.float32)

    def material(self, kind=MAT_DIFFUSE, albedo=(0.8, 0.8, 0.8), emission=(0, 0, 0), ior=1.5) -> int:
        self._mtypes.append(kind)
        self._mparams.append([*albedo, *emission, ior, 0.0])
        return len(self._mtypes) - 1

    def sphere(self, centre, radius, mat) -> int:
        self._types.append(PRIM_SPHERE)
        self._mats.append(mat)
        self._geom.append([*centre, radius, 0, 0, 0, 0, 0])
        return len(self._types) - 1

    def quad(self, centre, u, v, mat) -> int:
        self._types.append(PRIM_QUAD)
        self._mats.append(mat)
        self._geom.append([*centre, *u, *v])
        return len(self._types) - 1

    def box(self, centre, half, mat) -> int:
        self._types.append(PRIM_BOX)
        self._mats.append(mat)
        self._geom.append([*centre, *half, 0, 0, 0])
        return len(self._types) - 1

    def look_at(self, eye, look, up, vfov_deg):
        self.camera = np.array([*eye, *look, *up, vfov_deg], np.float32)

    def build(self) -> Scene:
        return Scene(
            prim_type=np.array(self._types, np.int32),
            prim_mat=np.array(self._mats, np.int32),
            prim_geom=np.array(self._geom, np.float32).reshape(-1, 9),
            mat_type=np.array(self._mtypes, np.int32),
            mat_param=np.array(self._mparams, np.float32).reshape(-1, 8),
            camera=self.camera.copy(),
            background=self.background.copy(),
        )


@dataclass
class Workload:
    name: str
    scene: Scene
    bindings: np.ndarray     # int32 [D, 3] (kind, index, component)
    theta_ref: np.ndarray    # float32 [D]
    theta0: np.ndarray       # float32 [D]
    sigma: np.ndarray        # float32 [D]
    width: int
    height: int
    spp: int
    depth: int
    rr_start: int            # first 0-based vertex index with Russian roulette; -1 = off
    pairs: int               # P antithetic pairs, R = 2P renders
    seed: int = 0
    lr: float = 1e-2
    steps: int = 100
    sampler: int = SAMPLER_RADIAL
    antithetic: int = 1
    crn: int = 1
    sigma_min: float = 0.01
    anneal: int = 0          # 1 = linear sigma decay after a warm start at 50 % of `steps`
    estimator: int = 0       # 0 = Eq. 10 (kernel-gradient weights), 1 = Eq. 9 (pathwise render gradients)
    extra: dict = field(default_factory=dict)

    @property
    def D(self) -> int:
        if self.bindings.shape[0] == 1 and int(self.bindings[0, 0]) == BIND_TEXTURE:
            return 3 * int(self.bindings[0, 2]) ** 2
        return int(self.bindings.shape[0])

    @property
    def renders(self) -> int:
        return 2 * self.pairs

    @property
    def paths_per_step(self) -> int:
        return self.renders * self.width * self.height * self.spp


def _f32(x):
    return np.asarray(x, np.float32)


def config_small(seed: int = 0) -> Workload:
    """64x64, one diffuse sphere (r = 0.5, albedo 0.8) on a diffuse ground plane, 0.5x0.5
    area light of radiance 10, depth 1 (direct light and shadow), 4 spp, theta = sphere
    centre xy, sigma = 0.1, 4 antithetic pairs (8 renders), Philox seed 0."""
    b = SceneBuilder()
    m_ground = b.material(MAT_DIFFUSE, (0.8, 0.8, 0.8))
    m_sphere = b.material(MAT_DIFFUSE, (0.8, 0.8, 0.8))
    m_light = b.material(MAT_DIFFUSE, (0.0, 0.0, 0.0), emission=(10.0, 10.0, 10.0))
    b.quad((0, 0, 0), (8, 0, 0), (0, 8, 0), m_ground)
    sph = b.sphere((0.0, 0.0, 0.5), 0.5, m_sphere)
    b.quad((1.5, 1.5, 2.5), (0.5, 0, 0), (0, -0.5, 0), m_light)
    b.look_at((0, 0, 5), (0, 0, 0), (0, 1, 0), 40.0)
    rng = np.random.default_rng(seed)
    theta0 = rng.uniform(-1.0, 1.0, size=2)
    return Workload(
        name="small-64x64-sphere-xy",
        scene=b.build(),
        bindings=np.array([[BIND_PRIM_POS, sph, 0], [BIND_PRIM_POS, sph, 1]], np.int32),
        theta_ref=_f32([0.3, -0.2]), theta0=_f32(theta0), sigma=_f32([0.1, 0.1]),
        width=64, height=64, spp=4, depth=1, rr_start=-1, pairs=4, seed=seed,
        lr=2e-2, steps=200,
    )


def config_occlusion(seed: int = 0) -> Workload:
    """256x256, three diffuse spheres and a 0.4^3 box on a plane under a 1x1 light,
    depth 4, 16 spp, theta = box centre (3-D), sigma = 0.05, N = 16 renders (P = 8)."""
    b = SceneBuilder()
    m_ground = b.material(MAT_DIFFUSE, (0.7, 0.7, 0.7))
    m_a = b.material(MAT_DIFFUSE, (0.85, 0.25, 0.2))
    m_b = b.material(MAT_DIFFUSE, (0.25, 0.8, 0.3))
    m_c = b.material(MAT_DIFFUSE, (0.25, 0.35, 0.85))
    m_box = b.material(MAT_DIFFUSE, (0.9, 0.8, 0.3))
    m_light = b.material(MAT_DIFFUSE, (0.0, 0.0, 0.0), emission=(15.0, 15.0, 15.0))
    b.quad((0, 0, 0), (16, 0, 0), (0, 16, 0), m_ground)
    b.sphere((-0.7, 0.4, 0.35), 0.35, m_a)
    b.sphere((0.75, 0.6, 0.3), 0.3, m_b)
    b.sphere((0.05, 1.1, 0.45), 0.45, m_c)
    box = b.box((0.0, 0.0, 0.2), (0.2, 0.2, 0.2), m_box)
    b.quad((0.0, 0.5, 3.0), (1, 0, 0), (0, -1, 0), m_light)
    b.look_at((0, -4.0, 2.5), (0, 0.5, 0.3), (0, 0, 1), 40.0)
    rng = np.random.default_rng(seed + 1)
    theta_ref = np.array([0.15, 0.35, 0.2])
    theta0 = theta_ref + np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(0.0, 0.3)])
    return Workload(
        name="occlusion-256x256-box-xyz",
        scene=b.build(),
        bindings=np.array([[BIND_PRIM_POS, box, 0], [BIND_PRIM_POS, box, 1], [BIND_PRIM_POS, box, 2]], np.int32),
        theta_ref=_f32(theta_ref), theta0=_f32(theta0), sigma=_f32([0.05, 0.05, 0.05]),
        width=256, height=256, spp=16, depth=4, rr_start=-1, pairs=8, seed=seed,
        lr=2e-2, steps=100,
    )


def config_gi_box(seed: int = 0) -> Workload:
    """512x512 open box of five diffuse walls (albedos U[0.2,0.9]^3, seeded), two boxes,
    one mirror sphere, ceiling light; depth 8 with Russian roulette from the 4th
    vertex; theta = light xyz + left and right wall RGB (D = 9); sigma0 = 0.125;
    N = 32 renders (P = 16), 32 spp, Adam lr 1e-2, 300 steps."""
    rng = np.random.default_rng(seed + 2)
    walls = rng.uniform(0.2, 0.9, size=(5, 3))
    b = SceneBuilder()
    mw = [b.material(MAT_DIFFUSE, tuple(walls[i])) for i in range(5)]
    m_box = b.material(MAT_DIFFUSE, (0.75, 0.75, 0.75))
    m_mirror = b.material(MAT_MIRROR, (0.9, 0.9, 0.9))
    m_light = b.material(MAT_DIFFUSE, (0.0, 0.0, 0.0), emission=(12.0, 12.0, 12.0))
    b.quad((0, 0, 0), (2, 0, 0), (0, 2, 0), mw[0])            # floor
    b.quad((0, 0, 2), (2, 0, 0), (0, -2, 0), mw[1])           # ceiling
    b.quad((0, 1, 1), (2, 0, 0), (0, 0, 2), mw[2])            # back
    b.quad((-1, 0, 1), (0, 2, 0), (0, 0, 2), mw[3])           # left
    b.quad((1, 0, 1), (0, 0, 2), (0, 2, 0), mw[4])            # right
    b.box((-0.4, 0.3, 0.6), (0.25, 0.25, 0.6), m_box)
    b.box((0.45, -0.2, 0.3), (0.3, 0.3, 0.3), m_box)
    b.sphere((0.5, 0.55, 0.25), 0.25, m_mirror)
    light = b.quad((0.0, 0.0, 1.98), (0.5, 0, 0), (0, -0.5, 0), m_light)
    b.look_at((0, -3.2, 1.0), (0, 0, 1.0), (0, 0, 1), 40.0)
    binds = [[BIND_PRIM_POS, light, c] for c in range(3)]
    binds += [[BIND_MAT_ALBEDO, mw[3], c] for c in range(3)]
    binds += [[BIND_MAT_ALBEDO, mw[4], c] for c in range(3)]
    theta_ref = np.array([0.1, 0.15, 1.95, 0.75, 0.2, 0.2, 0.2, 0.7, 0.25])
    theta0 = np.concatenate([[-0.3, -0.2, 1.9], walls[3], walls[4]])
    return Workload(
        name="gi-box-512x512-light-walls",
        scene=b.build(),
        bindings=np.array(binds, np.int32),
        theta_ref=_f32(theta_ref), theta0=_f32(theta0), sigma=_f32(np.full(9, 0.125)),
        width=512, height=512, spp=32, depth=8, rr_start=3, pairs=16, seed=seed,
        lr=1e-2, steps=300,
    )


def config_caustic(seed: int = 0) -> Workload:
    """512x512 glass sphere (IOR 1.5, r = 0.5, centre height 1) above a diffuse floor,
    0.2x0.2 light; depth 12 with Russian roulette from the 4th vertex;
    theta = light xyz; sigma0 = 0.125; N = 64 renders (P = 32), 64 spp."""
    b = SceneBuilder()
    m_floor = b.material(MAT_DIFFUSE, (0.8, 0.8, 0.8))
    m_glass = b.material(MAT_DIELECTRIC, (1.0, 1.0, 1.0), ior=1.5)
    m_light = b.material(MAT_DIFFUSE, (0.0, 0.0, 0.0), emission=(200.0, 200.0, 200.0))
    b.quad((0, 0, 0), (10, 0, 0), (0, 10, 0), m_floor)
    b.sphere((0.0, 0.0, 1.0), 0.5, m_glass)
    light = b.quad((0.6, 0.4, 2.6), (0.2, 0, 0), (0, -0.2, 0), m_light)
    b.look_at((0, -4.0, 1.2), (0, 0, 0.6), (0, 0, 1), 40.0)
    return Workload(
        name="caustic-512x512-light-xyz",
        scene=b.build(),
        bindings=np.array([[BIND_PRIM_POS, light, c] for c in range(3)], np.int32),
        theta_ref=_f32([0.6, 0.4, 2.6]), theta0=_f32([-0.4, -0.3, 2.3]), sigma=_f32([0.125] * 3),
        width=512, height=512, spp=64, depth=12, rr_start=3, pairs=32, seed=seed,
        lr=1e-2, steps=500,
    )


def config_small_albedo(seed: int = 0) -> Workload:
    """The small scene with material parameters instead: theta = sphere albedo RGB, ground
    albedo G and light emission R (D = 5); Gaussian perturbations (sigma 0.05 on the
    albedos, 2 on the emission) for the pathwise estimator of Eq. 9."""
    wl = config_small(seed)
    b = SceneBuilder()
    m_ground = b.material(MAT_DIFFUSE, (0.8, 0.8, 0.8))
    m_sphere = b.material(MAT_DIFFUSE, (0.8, 0.8, 0.8))
    m_light = b.material(MAT_DIFFUSE, (0.0, 0.0, 0.0), emission=(40.0, 40.0, 40.0))
    b.quad((0, 0, 0), (8, 0, 0), (0, 8, 0), m_ground)
    b.sphere((0.0, 0.0, 0.5), 0.5, m_sphere)
    b.quad((1.5, 1.5, 2.5), (0.5, 0, 0), (0, -0.5, 0), m_light)
    b.look_at((0, 0, 5), (0, 0, 0), (0, 1, 0), 40.0)
    rng = np.random.default_rng(seed + 5)
    theta_ref = np.array([0.7, 0.3, 0.4, 0.6, 30.0])
    theta0 = np.concatenate([rng.uniform(0.3, 0.9, size=4), [45.0]])
    binds = [[BIND_MAT_ALBEDO, m_sphere, c] for c in range(3)]
    binds += [[BIND_MAT_ALBEDO, m_ground, 1], [BIND_MAT_EMISSION, m_light, 0]]
    return Workload(
        name="small-64x64-albedo-emission", scene=b.build(), bindings=np.array(binds, np.int32),
        theta_ref=_f32(theta_ref), theta0=_f32(theta0), sigma=_f32([0.05, 0.05, 0.05, 0.05, 2.0]),
        width=wl.width, height=wl.height, spp=wl.spp, depth=wl.depth, rr_start=-1, pairs=4, seed=seed,
        lr=2e-2, steps=200, sampler=SAMPLER_GAUSS, estimator=1,
    )


def config_gi_albedo(seed: int = 0) -> Workload:
    """The GI box (512x512, depth 8 with Russian roulette from the 4th vertex, 32 spp,
    P = 16) with theta = left and right wall RGB albedo (D = 6), sigma = 0.125, for the
    pathwise estimator of Eq. 9 (Gaussian perturbations)."""
    wl = config_gi_box(seed)
    sl = slice(3, 9)
    return replace(wl, name="gi-box-512x512-walls-albedo", bindings=wl.bindings[sl].copy(),
                   theta_ref=wl.theta_ref[sl].copy(), theta0=wl.theta0[sl].copy(), sigma=wl.sigma[sl].copy(),
                   sampler=SAMPLER_GAUSS, estimator=1)


def config_texture(res: int = 128, px_per_texel: int = 2, seed: int = 0) -> Workload:
    """The paper's high-dimensional texture task (its supplemental "Compatibility"
    section) as an analytic stand-in: a res x res RGB texture (D = 3 res^2; 49,152 for
    res = 128) on a square diffuse plane seen straight from above under a uniform
    environment (background radiance 1), depth 2 (the plane, then the sky). The camera
    frames the plane exactly, px_per_texel pixels per texel side, so a pixel sees one
    texel and its value is that texel's albedo. theta_ref is a seeded smooth pattern in
    [0.2, 0.8], theta0 a uniform grey; sigma = 0.01 per texel; 8 pairs, 4 spp."""
    b = SceneBuilder()
    m_tex = b.material(MAT_DIFFUSE, (0.5, 0.5, 0.5))
    b.quad((0, 0, 0), (2, 0, 0), (0, -2, 0), m_tex)  # s along +x, t along -y: texel rows follow image rows
    b.look_at((0, 0, 1), (0, 0, 0), (0, 1, 0), 90.0)
    b.background = np.array([1.0, 1.0, 1.0], np.float32)
    rng = np.random.default_rng(seed + 11)
    y, x = np.mgrid[0:res, 0:res] / res
    ref = np.zeros((res, res, 3))
    for c in range(3):
        for _ in range(3):
            fx, fy, ph = rng.uniform(1.0, 4.0), rng.uniform(1.0, 4.0), rng.uniform(0, 2 * np.pi)
            ref[..., c] += np.sin(2 * np.pi * (fx * x + fy * y) + ph)
    ref = 0.5 + 0.3 * ref / np.abs(ref).max()
    D = 3 * res * res
    W = res * px_per_texel
    return Workload(
        name=f"texture-{res}x{res}-rgb", scene=b.build(),
        bindings=np.array([[BIND_TEXTURE, m_tex, res]], np.int32),
        theta_ref=_f32(ref.reshape(-1)), theta0=_f32(np.full(D, 0.5)), sigma=_f32(np.full(D, 0.01)),
        width=W, height=W, spp=4, depth=2, rr_start=-1, pairs=8, seed=seed, lr=1e-2, steps=300,
    )


def all_configs():
    return [config_small(), config_occlusion(), config_gi_box(), config_caustic()]


def scaled(w: Workload, width=None, height=None, spp=None, pairs=None, **kw) -> Workload:
    """Copy of `w` at a reduced size (used for parity cases the oracle finishes quickly)."""
    out = replace(w, scene=copy.deepcopy(w.scene))
    if width is not None:
        out.width = int(width)
    if height is not None:
        out.height = int(height)
    if spp is not None:
        out.spp = int(spp)
    if pairs is not None:
        out.pairs = int(pairs)
    for k, v in kw.items():
        setattr(out, k, v)
    return out


def serving_mix(n_jobs: int = 256, seed: int = 0, rate_hz: float | None = None):
    """Poisson stream of inverse-rendering jobs drawn uniformly from the first three
    workloads, each with its own resolution (128..512 in steps of 64), number of renders
    N in {8,16,32,64}, spp in {8,16,32,64}, reference and initial parameters.
    Returns a list of (arrival_time_s, Workload)."""
    rng = np.random.default_rng(seed + 100)
    makers = [config_small, config_occlusion, config_gi_box]
    jobs = []
    t = 0.0
    for j in range(n_jobs):
        base = makers[int(rng.integers(0, 3))](seed=int(rng.integers(0, 2**31 - 1)))
        res = int(rng.choice(np.arange(128, 513, 64)))
        n_renders = int(rng.choice([8, 16, 32, 64]))
        spp = int(rng.choice([8, 16, 32, 64]))
        wl = scaled(base, width=res, height=res, spp=spp, pairs=n_renders // 2)
        wl.seed = int(rng.integers(0, 2**31 - 1))
        wl.steps = 300 if base.name.startswith("gi-box") else 100
        # perturb the reference and the start point per job (positions +-0.2, albedos +-0.1)
        wl.theta_ref = (wl.theta_ref + rng.uniform(-0.1, 0.1, size=wl.D)).astype(np.float32)
        wl.theta0 = (wl.theta0 + rng.uniform(-0.1, 0.1, size=wl.D)).astype(np.float32)
        wl.name = f"job{j}-{base.name.split('-')[0]}-{res}-N{n_renders}-spp{spp}"
        if rate_hz:
            t += float(rng.exponential(1.0 / rate_hz))
        jobs.append((t, wl))
    return jobs
