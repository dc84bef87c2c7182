"""Pins of the oracle's high-dimensional parameter path (a texture of T x T RGB texels,
the paper's 49,152-dimensional texture task at reduced T).

* Texture lookup: a plane framed exactly by the camera under a uniform environment shows
  each texel's (clamped) albedo in exactly the pixels it covers (every path: plane, then
  sky; zero variance).
* The radial sampler in high dimension: per draw, sum_d w_d tau_d = c_D |tau| / sigma and
  sum_d w_d^2 = c_D^2 / sigma^2 (a unit direction); over draws, |tau|^2 / sigma^2 has the
  chi-square mean D + 1, E[w_d tau_d] = 1 and E[w_d tau_e] = 0 for d != e (so
  E[w tau^T] = I, the identity that makes Eq. 10 unbiased).
* The estimator on the texture: with the pixel-exact render the loss is a quadratic in
  theta, so each antithetic pair's (L+ - L-) / 2 equals grad L . tau exactly, and the
  estimate's projection on grad L averages to |grad L|^2.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def test_texture_plane_shows_each_texel_exactly():
    wl = workloads.config_texture(res=8, px_per_texel=2)
    theta = wl.theta_ref.copy()
    theta[:6] = [-0.5, 1.7, 0.25, 2.0, 0.0, 1.0]  # clamped at lookup
    img = oracle.render(wl.scene, wl.bindings, theta[None], wl.width, wl.height, 3, wl.depth, seed=5)[0]
    tex = np.clip(theta.reshape(8, 8, 3).astype(np.float64), 0.0, 1.0)
    assert np.array_equal(img, np.repeat(np.repeat(tex, 2, 0), 2, 1))


@pytest.mark.parametrize("D", [192, 3072])
def test_high_dimensional_radial_sampler(D):
    sigma = np.full(D, 0.02, np.float32)
    s = float(sigma[0])
    c = oracle.radial_constant(D)
    n = 300 if D > 1000 else 1500
    r2, diag, off = [], [], []
    for i in range(n):
        tau, _, w = oracle.sample(0, sigma, seed=9, step=1, index=i)
        r = math.sqrt(float((tau * tau).sum())) / s
        assert float((w * tau).sum()) == pytest.approx(c * r, rel=1e-12)
        assert float((w * w).sum()) == pytest.approx(c * c / (s * s), rel=1e-12)
        r2.append(r * r)
        diag.append(float((w * tau).sum()) / D)
        off.append(float((w * np.roll(tau, 1)).sum()) / D)
    r2, diag, off = np.array(r2), np.array(diag), np.array(off)
    assert abs(r2.mean() - (D + 1)) < 4.5 * math.sqrt(2.0 * (D + 1) / n)
    assert abs(diag.mean() - 1.0) < 4.5 * diag.std(ddof=1) / math.sqrt(n)
    assert abs(off.mean()) < 4.5 * off.std(ddof=1) / math.sqrt(n)


def test_texture_estimator_is_a_directional_derivative_per_pair():
    wl = workloads.config_texture(res=8, px_per_texel=2)
    wl.pairs = 400
    target = oracle.render_target(wl)
    theta = wl.theta0.astype(np.float64)
    k2 = 4.0  # pixels per texel
    grad_L = 2.0 * k2 / (3.0 * wl.width * wl.height) * (theta - wl.theta_ref.astype(np.float64))
    res = oracle.smoothed_grad(wl, target=target, step=3)
    taus = res["taus"].astype(np.float64)
    assert np.abs(taus).max() < 0.45  # theta +- tau stays inside [0, 1]: no clamping
    # the losses are the quadratic at the parameters the renderer got (FP32 sums theta + tau)
    th32 = (wl.theta0[None, :] + res["taus"]).astype(np.float64)
    quad = k2 / (3.0 * wl.width * wl.height) * ((th32 - wl.theta_ref.astype(np.float64)) ** 2).sum(1)
    np.testing.assert_allclose(res["losses"], quad, rtol=1e-12)
    # so each pair's half difference is the directional derivative along tau, up to the
    # FP32 rounding of theta +- tau
    half_diff = 0.5 * (res["losses"][0::2] - res["losses"][1::2])
    bound = 1e-5 * np.linalg.norm(grad_L) * np.linalg.norm(taus[0::2], axis=1)
    assert np.all(np.abs(half_diff - taus[0::2] @ grad_L) <= bound)
    # Eq. 10: g = (1/2P) sum_p w_p (L+ - L-); its projection on grad L has mean |grad L|^2
    proj = (res["weights"][0::2] * half_diff[:, None]) @ grad_L / (grad_L @ grad_L)
    se = proj.std(ddof=1) / math.sqrt(proj.size)
    assert abs(proj.mean() - 1.0) < 4.5 * se and se < 0.2
    assert float(res["grad"] @ grad_L / (grad_L @ grad_L)) == pytest.approx(proj.mean(), rel=1e-9)
