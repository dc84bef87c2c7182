"""FP64 CPU oracle of the plateau-reduced gradient estimator -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs of
`bench.py` may import this package. The CUDA library never does, and this package
never imports the CUDA library: the two share nothing except the scene data of
the `workloads` package.

Functions follow the paper (Fischer & Ritschel, "Plateau-reduced Differentiable
Path Tracing"):

* `philox_words`        -- Philox4x32-10 (Salmon et al. 2011), the uniform draws of Algorithm 1
* `sample_unit`, `sample` -- the perturbation sampler of Sec. 3.2 / Eq. 11 / supplemental ICDF
* `render`, `render_pixels` -- the Monte-Carlo forward model P(theta) of Eq. 1 / Eq. 3
* `mse`                 -- the image loss of Sec. 4.1
* `smoothed_grad`       -- Eq. 10 with the antithetic pairs of Algorithm 1
* `render_tangent`, `kdp_grad` -- Eq. 9: pathwise derivatives of the render for albedo and
                          emission parameters, and their mean over Gaussian perturbations
* `adam`                -- the optimiser of Sec. 3.4
* `sigma_schedule`      -- the linear bandwidth decay of Sec. 3.3

Parity pins (tests/test_oracle_*.py): Philox against curand's host generator and
published known answers; the sampler against its closed-form distribution; the
estimator against closed-form smoothed gradients and quadrature; the tracer
against the white furnace and analytic irradiance; the dielectric event (`dielectric`)
against the textbook Fresnel equations and Snell's law; Russian roulette against the
furnace mean; Adam against torch.optim.Adam. `library` runs the functions from a copy
of the oracle built with a planted mistake, to show that a pin catches it.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

TAG_PERTURB, TAG_PATH, TAG_TARGET = 1, 2, 3


class _SceneArrays(C.Structure):
    _fields_ = [
        ("n_prims", C.c_int), ("n_mats", C.c_int),
        ("prim_type", C.c_void_p), ("prim_mat", C.c_void_p), ("prim_geom", C.c_void_p),
        ("mat_type", C.c_void_p), ("mat_param", C.c_void_p),
        ("camera", C.c_void_p), ("background", C.c_void_p),
    ]


_LOSS_CB = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_float), C.c_int, C.c_int, C.c_void_p)


def _bind(L):
    """Argument and result types of the oracle's exported functions."""
    vp, i32, u32, u64, dbl = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_double
    L.orc_philox_fill.argtypes = [u64, u32, u32, u32, u32, i32, vp]
    L.orc_u01.argtypes = [u32]
    L.orc_u01.restype = dbl
    L.orc_sampler_uniforms.argtypes = [i32, i32]
    L.orc_sampler_uniforms.restype = i32
    L.orc_radial_constant.argtypes = [i32]
    L.orc_radial_constant.restype = dbl
    L.orc_sample_unit.argtypes = [i32, i32, vp, vp, vp]
    L.orc_sample.argtypes = [i32, i32, vp, u64, u32, u32, vp, vp, vp]
    L.orc_intersect.argtypes = [vp, i32, vp, vp, vp]
    L.orc_intersect.restype = dbl
    L.orc_dielectric.argtypes = [vp, vp, dbl, dbl, vp, vp, vp, vp]
    L.orc_dielectric.restype = i32
    L.orc_render.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, u64, u32, u32, i32, vp, i32]
    L.orc_render.restype = i32
    L.orc_render_pixels.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, u64, u32, u32, vp, i32, vp]
    L.orc_render_pixels.restype = i32
    L.orc_mse.argtypes = [vp, vp, i32, i32]
    L.orc_mse.restype = dbl
    L.orc_smoothed_grad.argtypes = [vp, vp, i32, vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32, u64,
                                    u32, vp, vp, vp, vp, vp, i32]
    L.orc_smoothed_grad.restype = i32
    L.orc_estimate.argtypes = [i32, i32, i32, vp, vp, i32, i32, u64, u32, _LOSS_CB, vp, vp, vp, vp, vp]
    L.orc_estimate.restype = i32
    L.orc_sample_unit_batch.argtypes = [i32, i32, i32, vp, vp, vp]
    L.orc_render_tangent.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, u64, u32, u32, vp, vp, i32]
    L.orc_render_tangent.restype = i32
    L.orc_kdp_grad.argtypes = [vp, vp, i32, vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, i32, u64, u32,
                               vp, vp, vp, vp, vp, i32]
    L.orc_kdp_grad.restype = i32
    L.orc_adam.argtypes = [i32, vp, vp, vp, vp, i32, dbl, dbl, dbl, dbl]
    L.orc_sigma_schedule.argtypes = [dbl, dbl, i32, i32]
    L.orc_sigma_schedule.restype = dbl
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(_build.build()))
    return _lib


@contextlib.contextmanager
def library(path: str):
    """Run the oracle's functions from another build of its source (the tests use this to
    plant a mistake in a copy of the oracle and check that a pin catches it)."""
    global _lib
    saved = lib()
    _lib = _bind(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _param_dim(binds: np.ndarray) -> int:
    """Parameters the bindings stand for: one per row, or 3 T^2 for a texture row (4, mat, T)."""
    binds = np.asarray(binds).reshape(-1, 3)
    if binds.shape[0] == 1 and int(binds[0, 0]) == 4:
        return 3 * int(binds[0, 2]) ** 2
    return binds.shape[0]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _SceneHandle:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, scene):
        self.arrays = [
            np.ascontiguousarray(scene.prim_type, np.int32), np.ascontiguousarray(scene.prim_mat, np.int32),
            np.ascontiguousarray(scene.prim_geom, np.float32), np.ascontiguousarray(scene.mat_type, np.int32),
            np.ascontiguousarray(scene.mat_param, np.float32), np.ascontiguousarray(scene.camera, np.float32),
            np.ascontiguousarray(scene.background, np.float32),
        ]
        a = self.arrays
        self.s = _SceneArrays(scene.n_prims, scene.n_mats, *[_ptr(x) for x in a])

    @property
    def ref(self):
        return C.byref(self.s)


def philox_words(seed: int, c1: int, c2: int, c3: int, c0_base: int, n: int) -> np.ndarray:
    """Philox4x32-10 words for counters (c0_base + i, c1, c2, c3), key = seed (lo, hi). [n, 4] uint32."""
    out = np.zeros((n, 4), np.uint32)
    lib().orc_philox_fill(seed, c1, c2, c3, c0_base, n, _ptr(out))
    return out


def u01(words: np.ndarray) -> np.ndarray:
    w = np.asarray(words, np.uint64)
    return ((w >> 9) * 2 + 1).astype(np.float64) / 16777216.0


def sampler_uniforms(mode: int, D: int) -> int:
    return int(lib().orc_sampler_uniforms(mode, D))


def radial_constant(D: int) -> float:
    return float(lib().orc_radial_constant(D))


def sample_unit(mode: int, D: int, u: np.ndarray):
    """Unit-bandwidth draw (tau~, w~) from explicit uniforms u (len >= sampler_uniforms)."""
    u = np.ascontiguousarray(u, np.float64)
    tau = np.zeros(D, np.float64)
    w = np.zeros(D, np.float64)
    lib().orc_sample_unit(mode, D, _ptr(u), _ptr(tau), _ptr(w))
    return tau, w


def sample_unit_batch(mode: int, D: int, u: np.ndarray):
    """Unit-bandwidth draws for a batch of uniform rows u [n, sampler_uniforms(mode, D)]."""
    nu = sampler_uniforms(mode, D)
    u = np.ascontiguousarray(u, np.float64).reshape(-1, nu)
    n = u.shape[0]
    tau = np.zeros((n, D), np.float64)
    w = np.zeros((n, D), np.float64)
    lib().orc_sample_unit_batch(mode, D, n, _ptr(u), _ptr(tau), _ptr(w))
    return tau, w


def estimate(loss, theta, sigma, pairs: int, mode: int = 0, antithetic: int = 1, seed: int = 0, step: int = 0,
             pair_begin: int = 0):
    """Eq. 10 estimate for an arbitrary Python loss L(theta_r: float32[D]) -> float.
    Returns dict(grad, losses, taus, weights)."""
    th = np.ascontiguousarray(theta, np.float32)
    sg = np.ascontiguousarray(sigma, np.float32)
    D = th.shape[0]

    def _cb(ptr, d, r, user):
        return float(loss(np.ctypeslib.as_array(ptr, shape=(d,)).copy()))

    cb = _LOSS_CB(_cb)
    grad = np.zeros(D, np.float64)
    losses = np.zeros(2 * pairs, np.float64)
    taus = np.zeros((2 * pairs, D), np.float32)
    weights = np.zeros((2 * pairs, D), np.float64)
    rc = lib().orc_estimate(mode, antithetic, D, _ptr(th), _ptr(sg), pairs, pair_begin, seed, step, cb, None,
                            _ptr(grad),
                            _ptr(losses), _ptr(taus), _ptr(weights))
    if rc:
        raise ValueError(f"oracle estimate failed ({rc})")
    return {"grad": grad, "losses": losses, "taus": taus, "weights": weights}


def sample(mode: int, sigma: np.ndarray, seed: int, step: int, index: int):
    """Draw `index` of `step`: (tau FP64, tau rounded to FP32, w FP64)."""
    sigma = np.ascontiguousarray(sigma, np.float32)
    D = sigma.shape[0]
    tau = np.zeros(D, np.float64)
    tf = np.zeros(D, np.float32)
    w = np.zeros(D, np.float64)
    lib().orc_sample(mode, D, _ptr(sigma), seed, step, index, _ptr(tau), _ptr(tf), _ptr(w))
    return tau, tf, w


def intersect(scene, prim: int, o, d):
    h = _SceneHandle(scene)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    n = np.zeros(3, np.float64)
    t = lib().orc_intersect(h.ref, prim, _ptr(o), _ptr(d), _ptr(n))
    return t, n


def dielectric(direction, normal, ior: float, u: float, point=(0.0, 0.0, 0.0)):
    """The tracer's smooth-dielectric event for one ray: direction (unit) meets a surface of
    index `ior` (outside index 1) with outward unit normal at `point`; u is the uniform of
    the reflect-or-refract choice. Returns dict(reflected, dir, org, F, rs, rp)."""
    d = np.ascontiguousarray(direction, np.float64)
    n = np.ascontiguousarray(normal, np.float64)
    p = np.ascontiguousarray(point, np.float64)
    nd, no, fr = np.zeros(3), np.zeros(3), np.zeros(3)
    refl = lib().orc_dielectric(_ptr(d), _ptr(n), float(ior), float(u), _ptr(p), _ptr(nd), _ptr(no), _ptr(fr))
    return {"reflected": bool(refl), "dir": nd, "org": no, "F": float(fr[0]), "rs": float(fr[1]), "rp": float(fr[2])}


def render(scene, bindings, thetas, width, height, spp, depth, rr_start=-1, seed=0, step=0, tag=TAG_PATH,
           crn=1, nthreads=0) -> np.ndarray:
    """Render n scenes at thetas [n, D] (FP32). Returns [n, H, W, 3] float64."""
    h = _SceneHandle(scene)
    binds = np.ascontiguousarray(bindings, np.int32).reshape(-1, 3)
    th = np.ascontiguousarray(np.atleast_2d(thetas), np.float32)
    n, D = th.shape
    if _param_dim(binds) != D:
        raise ValueError("thetas and bindings disagree on D")
    out = np.zeros((n, height, width, 3), np.float64)
    rc = lib().orc_render(h.ref, _ptr(binds), D, _ptr(th), n, width, height, spp, depth, rr_start, seed, step, tag,
                          crn, _ptr(out), nthreads)
    if rc:
        raise ValueError(f"oracle render failed ({rc})")
    return out


def render_pixels(scene, bindings, theta, pixels, width, height, spp, depth, rr_start=-1, seed=0, step=0,
                  tag=TAG_PATH, render_field=0) -> np.ndarray:
    """Selected pixels (linear indices) of one render. Returns [m, 3] float64."""
    h = _SceneHandle(scene)
    binds = np.ascontiguousarray(bindings, np.int32).reshape(-1, 3)
    th = np.ascontiguousarray(theta, np.float32)
    pix = np.ascontiguousarray(pixels, np.int32)
    out = np.zeros((pix.shape[0], 3), np.float64)
    rc = lib().orc_render_pixels(h.ref, _ptr(binds), th.shape[0], _ptr(th), render_field, width, height, spp, depth,
                                 rr_start, seed, step, tag, _ptr(pix), pix.shape[0], _ptr(out))
    if rc:
        raise ValueError(f"oracle render failed ({rc})")
    return out


def mse(image: np.ndarray, target: np.ndarray) -> float:
    img = np.ascontiguousarray(image, np.float64)
    tg = np.ascontiguousarray(target, np.float32)
    H, W = img.shape[0], img.shape[1]
    return float(lib().orc_mse(_ptr(img), _ptr(tg), W, H))


def smoothed_grad(wl, theta=None, sigma=None, target=None, step=0, pairs=None, mode=None, antithetic=None,
                  crn=None, nthreads=0, pair_begin=0):
    """Eq. 10 estimate at theta for workload `wl`. Returns dict(grad, losses, taus, weights)."""
    h = _SceneHandle(wl.scene)
    binds = np.ascontiguousarray(wl.bindings, np.int32)
    th = np.ascontiguousarray(wl.theta0 if theta is None else theta, np.float32)
    sg = np.ascontiguousarray(wl.sigma if sigma is None else sigma, np.float32)
    P = wl.pairs if pairs is None else pairs
    D = th.shape[0]
    tg = np.ascontiguousarray(target, np.float32)
    if tg.shape != (wl.height, wl.width, 4):
        raise ValueError("target must be [H, W, 4] float32")
    grad = np.zeros(D, np.float64)
    losses = np.zeros(2 * P, np.float64)
    taus = np.zeros((2 * P, D), np.float32)
    weights = np.zeros((2 * P, D), np.float64)
    rc = lib().orc_smoothed_grad(
        h.ref, _ptr(binds), D, _ptr(th), _ptr(sg), P, pair_begin, wl.sampler if mode is None else mode,
        wl.antithetic if antithetic is None else antithetic, wl.crn if crn is None else crn,
        wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, wl.seed, step, _ptr(tg),
        _ptr(grad), _ptr(losses), _ptr(taus), _ptr(weights), nthreads)
    if rc:
        raise ValueError(f"oracle smoothed_grad failed ({rc})")
    return {"grad": grad, "losses": losses, "taus": taus, "weights": weights}


def render_tangent(scene, bindings, theta, width, height, spp, depth, rr_start=-1, seed=0, step=0, tag=TAG_PATH,
                   render_field=0, nthreads=0):
    """One render at theta and its pathwise tangents (Eq. 9's dP/dtheta) for albedo and
    emission bindings: (image [H, W, 3], dimage [H, W, D]); dimage[..., d] is the
    derivative of channel bindings[d][2] of the pixel mean with respect to theta_d."""
    h = _SceneHandle(scene)
    binds = np.ascontiguousarray(bindings, np.int32)
    th = np.ascontiguousarray(theta, np.float32)
    D = th.shape[0]
    img = np.zeros((height, width, 3), np.float64)
    dimg = np.zeros((height, width, D), np.float64)
    rc = lib().orc_render_tangent(h.ref, _ptr(binds), D, _ptr(th), render_field, width, height, spp, depth,
                                  rr_start, seed, step, tag, _ptr(img), _ptr(dimg), nthreads)
    if rc:
        raise ValueError(f"oracle render_tangent failed ({rc})")
    return img, dimg


def kdp_grad(wl, theta=None, sigma=None, target=None, step=0, pairs=None, antithetic=None, crn=None, nthreads=0,
             pair_begin=0):
    """Eq. 9 estimate at theta (Gaussian draws, pathwise render gradients) for workload `wl`
    whose bindings are all albedo or emission ones. Returns dict(grad, losses, taus, rgrads)."""
    h = _SceneHandle(wl.scene)
    binds = np.ascontiguousarray(wl.bindings, np.int32)
    th = np.ascontiguousarray(wl.theta0 if theta is None else theta, np.float32)
    sg = np.ascontiguousarray(wl.sigma if sigma is None else sigma, np.float32)
    P = wl.pairs if pairs is None else pairs
    D = th.shape[0]
    tg = np.ascontiguousarray(target, np.float32)
    if tg.shape != (wl.height, wl.width, 4):
        raise ValueError("target must be [H, W, 4] float32")
    grad = np.zeros(D, np.float64)
    losses = np.zeros(2 * P, np.float64)
    taus = np.zeros((2 * P, D), np.float32)
    rgrads = np.zeros((2 * P, D), np.float64)
    rc = lib().orc_kdp_grad(
        h.ref, _ptr(binds), D, _ptr(th), _ptr(sg), P, pair_begin, wl.antithetic if antithetic is None else antithetic,
        wl.crn if crn is None else crn, wl.width, wl.height, wl.spp, wl.depth, wl.rr_start, wl.seed, step,
        _ptr(tg), _ptr(grad), _ptr(losses), _ptr(taus), _ptr(rgrads), nthreads)
    if rc:
        raise ValueError(f"oracle kdp_grad failed ({rc})")
    return {"grad": grad, "losses": losses, "taus": taus, "rgrads": rgrads}


def render_target(wl, nthreads=0) -> np.ndarray:
    """Target image of a workload: a render at theta_ref on stream TARGET, step 0, as [H, W, 4] float32."""
    img = render(wl.scene, wl.bindings, wl.theta_ref[None, :], wl.width, wl.height, wl.spp, wl.depth, wl.rr_start,
                 wl.seed, 0, TAG_TARGET, 1, nthreads)[0]
    out = np.zeros((wl.height, wl.width, 4), np.float32)
    out[..., :3] = img
    return out


def adam(theta, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t is 1-based) in FP64; returns new (theta, m, v)."""
    th = np.array(theta, np.float64)
    mm = np.array(m, np.float64)
    vv = np.array(v, np.float64)
    gg = np.ascontiguousarray(g, np.float64)
    lib().orc_adam(th.shape[0], _ptr(th), _ptr(mm), _ptr(vv), _ptr(gg), t, lr, b1, b2, eps)
    return th, mm, vv


def sigma_schedule(sigma0: float, sigma_min: float, t: int, total: int) -> float:
    return float(lib().orc_sigma_schedule(sigma0, sigma_min, t, total))
