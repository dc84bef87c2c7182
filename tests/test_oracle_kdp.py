"""Pins of the oracle's pathwise estimator (Eq. 9, kappa-dP) for albedo and emission
parameters.

* The render tangents are the exact derivatives of the pixel means for fixed random
  numbers: with the perturbed parameters bound to materials and no Russian roulette, a
  pixel mean is a polynomial of degree <= depth in each parameter, so a five-point
  central difference over FP32-exact stencil points reproduces it to rounding.
* The per-render loss gradient is the derivative of the rendered image loss (same check
  on the loss).
* Russian roulette keeps the derivative unbiased: with the survival probability held
  constant in the derivative, the mean tangent over many paths equals the mean tangent
  without roulette (statistical).
* In expectation over the Gaussian kernel the estimator is the gradient of the smoothed
  objective: Gauss-Hermite quadrature of the pathwise gradient equals the five-point
  difference of the Gauss-Hermite smoothed loss (the loss is a quartic in the floor's
  albedo, so the difference is exact), and the sampled estimator converges to it.
"""
import math

import numpy as np
import pytest
from scipy.special import roots_hermite

import oracle
import workloads
from workloads import BIND_MAT_ALBEDO, MAT_DIFFUSE, SceneBuilder, Workload


def _small(depth, rr_start=-1, w=12, h=10, spp=2):
    wl = workloads.scaled(workloads.config_small_albedo(), width=w, height=h, spp=spp)
    wl.depth, wl.rr_start = depth, rr_start
    return wl


# FP32-exact parameters and steps: every stencil point is representable, so the
# difference quotient sees the same renders as the tangent's parameters.
THETA = np.array([0.5, 0.375, 0.625, 0.25, 32.0], np.float32)
STEPS = np.array([2.0 ** -5, 2.0 ** -5, 2.0 ** -5, 2.0 ** -5, 2.0], np.float64)


def _fd5(f, theta, d, h):
    e = np.zeros_like(theta)
    e[d] = h
    return (8 * (f(theta + e) - f(theta - e)) - (f(theta + 2 * e) - f(theta - 2 * e))) / (12 * h)


@pytest.mark.parametrize("depth", [1, 3])
def test_render_tangent_matches_fd_of_pixel_means(depth):
    wl = _small(depth)
    img, dimg = oracle.render_tangent(wl.scene, wl.bindings, THETA, wl.width, wl.height, wl.spp, wl.depth,
                                      seed=wl.seed, step=3)

    def render(th):
        return oracle.render(wl.scene, wl.bindings, np.asarray(th, np.float32)[None], wl.width, wl.height, wl.spp,
                             wl.depth, seed=wl.seed, step=3)[0]

    assert np.array_equal(img, render(THETA))
    for d in range(wl.D):
        fd = _fd5(lambda t: render(t), THETA.astype(np.float64), d, STEPS[d])
        c = int(wl.bindings[d, 2])
        scale = np.abs(fd[..., c]).max()
        assert scale > 0
        np.testing.assert_allclose(dimg[..., d], fd[..., c], rtol=0, atol=1e-9 * scale + 1e-12)
        for other in set(range(3)) - {c}:  # a channel's parameter changes no other channel
            assert np.abs(fd[..., other]).max() <= 1e-9 * scale + 1e-12


@pytest.mark.parametrize("depth", [1, 3])
def test_loss_gradient_matches_fd_of_render_loss(depth):
    wl = _small(depth)
    target = oracle.render_target(workloads.scaled(wl))
    zero = np.zeros(wl.D, np.float32)  # sigma = 0: every render sits at theta itself
    res = oracle.kdp_grad(wl, theta=THETA, sigma=zero, target=target, pairs=1, step=2)
    assert np.array_equal(res["rgrads"][0], res["rgrads"][1])  # common random numbers

    def loss(th):
        im = oracle.render(wl.scene, wl.bindings, np.asarray(th, np.float32)[None], wl.width, wl.height, wl.spp,
                           wl.depth, seed=wl.seed, step=2)[0]
        return oracle.mse(im, target)

    for d in range(wl.D):  # pixel means of degree <= 2 per parameter: a quartic loss
        fd = _fd5(loss, THETA.astype(np.float64), d, STEPS[d])
        assert res["rgrads"][0, d] == pytest.approx(fd, rel=1e-9, abs=1e-14)
    assert res["losses"][0] == pytest.approx(loss(THETA), rel=1e-15)


def test_russian_roulette_keeps_the_derivative_unbiased():
    wl = _small(4, w=4, h=4, spp=256)
    means = {}
    for rr in (-1, 0):
        per_seed = []
        for seed in range(16):
            _, dimg = oracle.render_tangent(wl.scene, wl.bindings, THETA, wl.width, wl.height, wl.spp, wl.depth,
                                            rr_start=rr, seed=100 + seed)
            per_seed.append(dimg.mean(axis=(0, 1)))
        per_seed = np.array(per_seed)
        means[rr] = (per_seed.mean(0), per_seed.std(0, ddof=1) / math.sqrt(len(per_seed)))
    (m0, s0), (m1, s1) = means[-1], means[0]
    se = np.sqrt(s0 ** 2 + s1 ** 2)
    assert np.all(np.abs(m0 - m1) < 4.5 * se), (m0, m1, se)
    assert np.all(se < 0.2 * np.abs(m0))  # the check has power


def _floor_workload(seed=4):
    """8x8 view of a diffuse sphere on a diffuse floor under a quad light; theta = the
    floor's red albedo. Depth 3, no Russian roulette: a path meets the floor at most twice
    (floor, sphere, floor), so a pixel mean is quadratic and the loss quartic in theta."""
    b = SceneBuilder()
    m_floor = b.material(MAT_DIFFUSE, (0.6, 0.6, 0.6))
    m_sph = b.material(MAT_DIFFUSE, (0.5, 0.5, 0.5))
    m_l = b.material(MAT_DIFFUSE, (0, 0, 0), emission=(20, 20, 20))
    b.quad((0, 0, 0), (8, 0, 0), (0, 8, 0), m_floor)
    b.sphere((0, 0, 0.5), 0.5, m_sph)
    b.quad((0.8, 0.8, 2.5), (0.5, 0, 0), (0, -0.5, 0), m_l)
    b.look_at((0, -3, 2), (0, 0, 0.4), (0, 0, 1), 40.0)
    return Workload(name="floor-albedo-r", scene=b.build(),
                    bindings=np.array([[BIND_MAT_ALBEDO, m_floor, 0]], np.int32),
                    theta_ref=np.array([0.8], np.float32), theta0=np.array([0.375], np.float32),
                    sigma=np.array([0.015], np.float32), width=8, height=8, spp=2, depth=3, rr_start=-1, pairs=2,
                    seed=seed, sampler=workloads.SAMPLER_GAUSS, estimator=1)


def test_kdp_expectation_is_the_smoothed_gradient():
    wl = _floor_workload()
    target = oracle.render_target(wl)
    theta, sigma = float(wl.theta0[0]), float(wl.sigma[0])
    x, wq = roots_hermite(12)
    # FP32 nodes in [0.25, 0.5): every node plus a multiple of 2^-6 stays FP32-exact, so
    # the smoothed loss below is evaluated at exactly the shifted nodes
    nodes = np.float32(theta + math.sqrt(2.0) * sigma * x)
    assert nodes.min() - 2 * 2.0 ** -6 >= 0.25 and nodes.max() + 2 * 2.0 ** -6 < 0.5

    def grad_at(t):  # the oracle's per-render loss gradient at theta = t (sigma = 0)
        res = oracle.kdp_grad(wl, theta=np.array([t], np.float32), sigma=np.zeros(1, np.float32), target=target,
                              pairs=1)
        return res["rgrads"][0, 0]

    def loss_at(t):
        im = oracle.render(wl.scene, wl.bindings, np.array([[t]], np.float32), wl.width, wl.height, wl.spp,
                           wl.depth, seed=wl.seed)[0]
        return oracle.mse(im, target)

    expect = float((wq * np.array([grad_at(t) for t in nodes])).sum() / math.sqrt(math.pi))

    def smoothed(t):
        shift = t[0] - theta
        return float((wq * np.array([loss_at(n + shift) for n in nodes.astype(np.float64)])).sum()
                     / math.sqrt(math.pi))

    fd = _fd5(smoothed, np.array([theta]), 0, 2.0 ** -6)
    assert expect == pytest.approx(fd, rel=1e-9)
    # not the plain gradient at theta: the smoothing matters for this loss
    assert abs(expect - grad_at(np.float32(theta))) > 1e-6 * abs(expect)

    # the sampled estimator (Gaussian draws, antithetic pairs) converges to it
    P = 400
    res = oracle.kdp_grad(wl, target=target, pairs=P)
    pair_means = 0.5 * (res["rgrads"][0::2, 0] + res["rgrads"][1::2, 0])
    se = pair_means.std(ddof=1) / math.sqrt(P)
    assert abs(res["grad"][0] - expect) < 4.5 * se
    assert se < 0.1 * abs(expect)


def test_kdp_rejects_geometry_bindings():
    wl = workloads.scaled(workloads.config_small(), width=8, height=8, spp=1)
    target = np.zeros((8, 8, 4), np.float32)
    with pytest.raises(ValueError):
        oracle.kdp_grad(wl, target=target, pairs=1)
