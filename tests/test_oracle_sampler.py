"""Pins of the oracle's perturbation sampler and estimator (Sec. 3.2, Eq. 10, Eq. 11,
Algorithm 1, supplemental ICDF derivation) against closed forms.

* The 1-D positivized kernel gradient |d kappa/d tau| normalised over the real
  line is |tau| exp(-tau^2/2s^2)/(2s^2); its CDF (signs as the supplemental's
  continuity argument requires) is F = exp(-t^2/2)/2 for t<0, 1-exp(-t^2/2)/2 else.
* The radial D-dim sampler: radius ~ chi with D+1 degrees of freedom, direction
  uniform on the sphere, weight norm c_D = E|N(0, I_D)|.
* For L = H(theta - a) (a plateau everywhere but at a), the Gaussian-smoothed
  loss is Phi((theta-a)/sigma) with derivative phi((theta-a)/sigma)/sigma.
* For a quadratic L the smoothed gradient equals the plain gradient.
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import gammaln

import oracle

RADIAL, PERDIM, GAUSS = 0, 1, 2


def _uniforms(n, nu, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(1e-12, 1.0, size=(n, nu))


def _two_sided_rayleigh_cdf(t):
    t = np.asarray(t)
    return np.where(t < 0, 0.5 * np.exp(-0.5 * t * t), 1.0 - 0.5 * np.exp(-0.5 * t * t))


@pytest.mark.parametrize("mode", [RADIAL, PERDIM])
def test_1d_sampler_follows_positivized_kernel_gradient(mode):
    nu = oracle.sampler_uniforms(mode, 1)
    tau, w = oracle.sample_unit_batch(mode, 1, _uniforms(200_000, nu, 1))
    ks = stats.kstest(tau[:, 0], _two_sided_rayleigh_cdf)
    assert ks.pvalue > 1e-3
    # E|tau| = sqrt(pi/2) for the two-sided Rayleigh
    m = np.abs(tau[:, 0]).mean()
    se = np.abs(tau[:, 0]).std() / math.sqrt(tau.shape[0])
    assert abs(m - math.sqrt(math.pi / 2)) < 4 * se
    # weight = sign(tau) * sqrt(2/pi): the half-space normalisation of |kappa'|
    assert np.allclose(w[:, 0], np.sign(tau[:, 0]) * math.sqrt(2 / math.pi), rtol=0, atol=1e-15)


def test_1d_radial_is_algorithm_1_magnitude():
    # Algorithm 1: tau = sqrt(-2 sigma^2 log xi); the first uniform is xi, the second the sign
    xi = np.array([0.1, 0.5 + 2 ** -24, 0.9, 1e-6])
    for x in xi:
        for s_u, s in [(0.25, -1.0), (0.75, 1.0)]:
            tau, w = oracle.sample_unit(RADIAL, 1, np.array([x, s_u]))
            assert tau[0] == pytest.approx(s * math.sqrt(-2 * math.log(x)), rel=1e-15)
            assert w[0] == pytest.approx(s * math.sqrt(2 / math.pi), rel=1e-15)


def test_perdim_inverse_cdf_closed_form():
    # F^-1(xi) = -sqrt(-2 ln 2xi) for xi < 1/2 and +sqrt(-2 ln 2(1-xi)) otherwise
    for xi in [1e-7, 0.1, 0.3, 0.5 - 2 ** -24, 0.5 + 2 ** -24, 0.7, 0.999]:
        tau, _ = oracle.sample_unit(PERDIM, 1, np.array([xi]))
        assert _two_sided_rayleigh_cdf(tau[0]) == pytest.approx(xi, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 9, 16, 64])
def test_radial_constant_is_mean_gaussian_norm(D):
    c = oracle.radial_constant(D)
    assert c == pytest.approx(math.sqrt(2) * math.exp(gammaln((D + 1) / 2) - gammaln(D / 2)), rel=1e-13)
    known = {1: math.sqrt(2 / math.pi), 2: math.sqrt(math.pi / 2), 3: 2 * math.sqrt(2 / math.pi)}
    if D in known:
        assert c == pytest.approx(known[D], rel=1e-14)


@pytest.mark.parametrize("D", [2, 3, 4, 9])
def test_radial_sampler_distribution(D):
    nu = oracle.sampler_uniforms(RADIAL, D)
    tau, w = oracle.sample_unit_batch(RADIAL, D, _uniforms(60_000, nu, D))
    r = np.linalg.norm(tau, axis=1)
    assert stats.kstest(r, stats.chi(D + 1).cdf).pvalue > 1e-3
    u = tau / r[:, None]
    # weight = c_D * direction
    assert np.allclose(w, oracle.radial_constant(D) * u, rtol=1e-12, atol=1e-14)
    # direction uniform on S^{D-1}: mean 0, second moment I/D
    n = u.shape[0]
    assert np.all(np.abs(u.mean(0)) < 5 / math.sqrt(n * D))
    cov = u.T @ u / n
    assert np.allclose(cov, np.eye(D) / D, atol=6 / math.sqrt(n) / D + 2e-3)
    if D == 3:  # Archimedes: a coordinate of a uniform point on S^2 is U[-1, 1]
        assert stats.kstest(u[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-3


@pytest.mark.parametrize("D", [1, 2, 5])
def test_gauss_sampler_is_standard_normal(D):
    nu = oracle.sampler_uniforms(GAUSS, D)
    tau, w = oracle.sample_unit_batch(GAUSS, D, _uniforms(60_000, nu, 10 + D))
    for d in range(D):
        assert stats.kstest(tau[:, d], stats.norm.cdf).pvalue > 1e-3
    assert np.array_equal(tau, w)


@pytest.mark.parametrize("mode", [RADIAL, PERDIM])
def test_step_function_smoothed_gradient_by_quadrature(mode):
    """Deterministic pin: integrate the pair estimator over its uniform (midpoint
    rule, 10^6 nodes) for L = H(theta - a); it must equal phi((theta-a)/s)/s."""
    sigma, a = 0.3, 0.2
    n = 1_000_000
    xi = (np.arange(n) + 0.5) / n
    if mode == RADIAL:
        u = np.stack([xi, np.full(n, 0.75)], 1)
    else:
        u = xi[:, None]
    tau_t, w_t = oracle.sample_unit_batch(mode, 1, u)
    tau = sigma * tau_t[:, 0]
    w = w_t[:, 0] / sigma
    for theta in [-0.4, 0.0, 0.15, 0.2, 0.5, 1.2]:
        pair = 0.5 * w * ((theta + tau - a > 0).astype(float) - (theta - tau - a > 0).astype(float))
        expect = stats.norm.pdf((theta - a) / sigma) / sigma
        # the integrand is a step in xi: the midpoint rule errs by at most |w|/n absolute
        assert pair.mean() == pytest.approx(expect, rel=2e-5, abs=float(np.abs(w).max()) / n)


@pytest.mark.parametrize("mode", [RADIAL, PERDIM, GAUSS])
@pytest.mark.parametrize("antithetic", [1, 0])
def test_estimator_unbiased_on_step(mode, antithetic):
    sigma, a, theta = 0.25, 0.1, -0.05
    res = oracle.estimate(lambda th: float(th[0] - a > 0), [theta], [sigma], pairs=20_000, mode=mode,
                          antithetic=antithetic, seed=11)
    L, w = res["losses"], res["weights"][:, 0]
    contrib = (w[0::2] * (L[0::2] - L[1::2]) / 2) if antithetic else (w * L)
    se = contrib.std() / math.sqrt(contrib.size)
    expect = stats.norm.pdf((theta - a) / sigma) / sigma
    assert abs(res["grad"][0] - expect) < 4.5 * se


@pytest.mark.parametrize("mode", [RADIAL, PERDIM, GAUSS])
@pytest.mark.parametrize("D", [1, 2, 3, 9])
def test_estimator_unbiased_on_quadratic(mode, D):
    rng = np.random.default_rng(100 + D)
    Q = rng.normal(size=(D, D))
    A = Q @ Q.T + D * np.eye(D)
    theta_star = rng.normal(size=D)
    theta = rng.normal(size=D).astype(np.float32)
    sigma = rng.uniform(0.05, 0.3, size=D).astype(np.float32)

    def L(th):
        e = th.astype(np.float64) - theta_star
        return 0.5 * e @ A @ e

    P = 4000
    res = oracle.estimate(L, theta, sigma, pairs=P, mode=mode, seed=5 + D)
    per_pair = res["weights"][0::2] * (res["losses"][0::2] - res["losses"][1::2])[:, None] / 2
    se = per_pair.std(0) / math.sqrt(P)
    expect = A @ (theta.astype(np.float64) - theta_star)
    assert np.all(np.abs(res["grad"] - expect) < 4.5 * se + 1e-9)


def test_nonseparable_step_radial_unbiased_perdim_not():
    """H(theta1 + theta2 - a) smoothed by N(0, s^2 I): d/dtheta_d = phi(x/(s sqrt2))/(s sqrt2).
    The radial sampler is unbiased in any D; the literal per-dimension sampler is not."""
    s, a = 0.3, 0.2
    theta = np.array([0.1, -0.05], np.float32)
    x = float(theta.sum()) - a
    expect = stats.norm.pdf(x / (s * math.sqrt(2))) / (s * math.sqrt(2))
    loss = lambda th: float(th[0] + th[1] - a > 0)  # noqa: E731
    res = oracle.estimate(loss, theta, [s, s], pairs=100_000, mode=RADIAL, seed=3)
    per_pair = res["weights"][0::2] * (res["losses"][0::2] - res["losses"][1::2])[:, None] / 2
    se = per_pair.std(0) / math.sqrt(per_pair.shape[0])
    assert np.all(np.abs(res["grad"] - expect) < 4.5 * se)
    res_pd = oracle.estimate(loss, theta, [s, s], pairs=100_000, mode=PERDIM, seed=3)
    assert np.all(np.abs(res_pd["grad"] - expect) > 0.1 * expect)


def test_constant_loss_gives_exact_zero():
    for mode in (RADIAL, PERDIM, GAUSS):
        res = oracle.estimate(lambda th: 0.125, [0.3, -0.2, 0.7], [0.1, 0.2, 0.3], pairs=64, mode=mode)
        assert np.all(res["grad"] == 0.0)


def test_antithetic_structure_and_fp32_perturbations():
    theta = np.array([0.3, -0.2], np.float32)
    sigma = np.array([0.1, 0.05], np.float32)
    seen = []
    res = oracle.estimate(lambda th: seen.append(th.copy()) or 0.0, theta, sigma, pairs=8, seed=9, step=4)
    taus, w = res["taus"], res["weights"]
    assert np.array_equal(taus[1::2], -taus[0::2]) and np.array_equal(w[1::2], -w[0::2])
    for r in range(16):
        assert np.array_equal(seen[r], (theta + taus[r]).astype(np.float32))
    # draw p of step t depends only on (seed, t, p): re-drawing it directly agrees
    for p in range(8):
        tau64, tau32, w64 = oracle.sample(RADIAL, sigma, 9, 4, p)
        assert np.array_equal(taus[2 * p], tau32) and np.allclose(w[2 * p], w64, rtol=0, atol=0)
    # another step draws different perturbations
    assert not np.array_equal(oracle.sample(RADIAL, sigma, 9, 5, 0)[1], taus[0])


def test_sigma_scales_tau_and_weight():
    u = _uniforms(1, oracle.sampler_uniforms(RADIAL, 3), 7)[0]
    tt, wt = oracle.sample_unit(RADIAL, 3, u)
    # linear scaling with sigma: tau = sigma * tau~, w = w~ / sigma (per dimension)
    for p in range(4):
        tau, _, w = oracle.sample(RADIAL, np.array([0.1, 0.2, 0.4], np.float32), 0, 0, p)
        tau2, _, w2 = oracle.sample(RADIAL, np.array([0.2, 0.4, 0.8], np.float32), 0, 0, p)
        assert np.allclose(tau2, 2 * tau, rtol=1e-14) and np.allclose(w2, w / 2, rtol=1e-14)
    assert np.linalg.norm(wt) == pytest.approx(oracle.radial_constant(3), rel=1e-14)
