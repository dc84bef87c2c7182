"""End-to-end pins of the oracle's estimator on real renders, and of its optimiser.

* Common random numbers: a parameter that changes no path (an object nobody sees,
  that blocks no light) gets a gradient of exactly zero, because both renders of
  each antithetic pair trace identical paths.
* Brute-force finite differences of the smoothed objective: on a tiny scene whose
  parameters are albedos, the loss of a fixed set of paths is a polynomial in
  theta, so Gauss-Hermite quadrature gives L_sigma(theta +- h) exactly and its
  central difference is the smoothed gradient; the oracle's Eq. 10 estimator must
  agree in expectation (many pairs, within 4.5 standard errors), and a
  generalised Gauss-Laguerre quadrature of its 1-D sampler must agree to 2e-6
  (the FP32 rounding of the rendered parameters).
* Adam against torch.optim.Adam (float64) on the same gradient sequence.
* The bandwidth schedule (Sec. 3.3 plus the supplemental's 50 % warm start).
"""
import math

import numpy as np
import pytest
from scipy.special import roots_genlaguerre, roots_hermite

import oracle
import workloads
from workloads import BIND_MAT_ALBEDO, BIND_PRIM_POS, MAT_DIFFUSE, SceneBuilder, Workload


def _with_far_sphere(wl):
    """Add a tiny sphere far away (out of view, in no light path) and bind its x."""
    sc = wl.scene
    sc.prim_geom = np.vstack([sc.prim_geom, [[50.0, 50.0, 50.0, 0.05, 0, 0, 0, 0, 0]]]).astype(np.float32)
    sc.prim_type = np.append(sc.prim_type, 0).astype(np.int32)
    sc.prim_mat = np.append(sc.prim_mat, 0).astype(np.int32)
    return sc.n_prims - 1


def test_invisible_parameter_gets_exact_zero_under_crn():
    """With only invisible parameters perturbed, both renders of every pair trace the
    same paths in the same scene, so L+ == L- bit for bit and the gradient is exactly 0."""
    wl = workloads.scaled(workloads.config_small(), width=24, height=24, spp=2, pairs=6)
    far = _with_far_sphere(wl)
    wl.bindings = np.array([[BIND_PRIM_POS, far, 0]], np.int32)
    wl.theta0 = wl.theta_ref = np.array([50.0], np.float32)
    wl.sigma = np.array([0.1], np.float32)
    target = oracle.render_target(wl)
    res = oracle.smoothed_grad(wl, target=target, crn=1)
    assert res["grad"][0] == 0.0 and np.all(res["losses"][0::2] == res["losses"][1::2])
    # without common random numbers the same parameter picks up pure noise
    res2 = oracle.smoothed_grad(wl, target=target, crn=0)
    assert res2["grad"][0] != 0.0


def test_invisible_parameter_is_zero_in_expectation_when_perturbed_jointly():
    """Perturbed together with visible parameters, an invisible one still gets a
    per-pair weight times the visible loss difference: zero only in expectation."""
    wl = workloads.scaled(workloads.config_small(), width=16, height=16, spp=1, pairs=400)
    far = _with_far_sphere(wl)
    wl.bindings = np.vstack([wl.bindings, [[BIND_PRIM_POS, far, 0]]]).astype(np.int32)
    wl.theta0 = np.append(wl.theta0, 50.0).astype(np.float32)
    wl.theta_ref = np.append(wl.theta_ref, 50.0).astype(np.float32)
    wl.sigma = np.append(wl.sigma, 0.1).astype(np.float32)
    target = oracle.render_target(wl)
    res = oracle.smoothed_grad(wl, target=target)
    per_pair = res["weights"][0::2] * (res["losses"][0::2] - res["losses"][1::2])[:, None] / 2
    se = per_pair.std(0) / math.sqrt(per_pair.shape[0])
    assert res["grad"][2] != 0.0 and abs(res["grad"][2]) < 4.5 * se[2]


def _albedo_scene():
    """8x8 view of a diffuse sphere on a diffuse floor under a quad light; theta binds
    the sphere's red and green albedo. Depth 2, no Russian roulette: the loss of fixed
    paths is a polynomial (degree <= 4) in theta."""
    b = SceneBuilder()
    m_floor = b.material(MAT_DIFFUSE, (0.6, 0.6, 0.6))
    m_sph = b.material(MAT_DIFFUSE, (0.5, 0.5, 0.5))
    m_l = b.material(MAT_DIFFUSE, (0, 0, 0), emission=(20, 20, 20))
    b.quad((0, 0, 0), (8, 0, 0), (0, 8, 0), m_floor)
    b.sphere((0, 0, 0.5), 0.5, m_sph)
    b.quad((0.8, 0.8, 2.5), (0.5, 0, 0), (0, -0.5, 0), m_l)
    b.look_at((0, -3, 2), (0, 0, 0.4), (0, 0, 1), 40.0)
    binds = np.array([[BIND_MAT_ALBEDO, m_sph, 0], [BIND_MAT_ALBEDO, m_sph, 1]], np.int32)
    return b.build(), binds


def _tiny_workload(D):
    sc, binds = _albedo_scene()
    binds = binds[:D]
    return Workload(name="albedo", scene=sc, bindings=binds, theta_ref=np.array([0.8, 0.2][:D], np.float32),
                    theta0=np.array([0.45, 0.55][:D], np.float32), sigma=np.array([0.06, 0.05][:D], np.float32),
                    width=8, height=8, spp=2, depth=2, rr_start=-1, pairs=2, seed=4)


def _loss_fn(wl, target):
    def L(thetas):
        th = np.atleast_2d(thetas).astype(np.float32)
        imgs = oracle.render(wl.scene, wl.bindings, th, wl.width, wl.height, wl.spp, wl.depth, wl.rr_start,
                             wl.seed, 0, oracle.TAG_PATH, 1)
        return np.array([oracle.mse(im, target) for im in imgs])
    return L


def _smoothed_loss_gh(L, theta, sigma, n=24):
    """L_sigma(theta) = E_{tau ~ N(0, sigma^2 I)} L(theta + tau) by tensor Gauss-Hermite."""
    x, wq = roots_hermite(n)
    D = len(theta)
    grids = np.meshgrid(*([x] * D), indexing="ij")
    wgrid = np.prod(np.meshgrid(*([wq] * D), indexing="ij"), axis=0).reshape(-1)
    pts = np.stack([g.reshape(-1) for g in grids], 1)
    th = theta[None, :] + math.sqrt(2.0) * sigma[None, :] * pts
    return float((wgrid * L(th)).sum() / math.pi ** (D / 2))


def _fd5(f, theta, d, h=0.04):
    """Five-point central difference along d: exact for polynomials of degree <= 4,
    and h large enough that FP32 rounding of the rendered parameters does not matter."""
    e = np.zeros_like(theta)
    e[d] = h
    return (8 * (f(theta + e) - f(theta - e)) - (f(theta + 2 * e) - f(theta - 2 * e))) / (12 * h)


@pytest.mark.parametrize("D", [1, 2])
def test_estimator_matches_fd_of_smoothed_objective(D):
    wl = _tiny_workload(D)
    target = oracle.render_target(wl)
    L = _loss_fn(wl, target)
    theta = wl.theta0.astype(np.float64)
    sigma = wl.sigma.astype(np.float64)
    fd = np.array([_fd5(lambda t: _smoothed_loss_gh(L, t, sigma), theta, d) for d in range(D)])
    # the oracle's estimator, end to end (sampler + FP32 perturbation + render + loss + reduction)
    P = 1500
    res = oracle.smoothed_grad(wl, target=target, pairs=P)
    per_pair = res["weights"][0::2] * (res["losses"][0::2] - res["losses"][1::2])[:, None] / 2
    se = per_pair.std(0) / math.sqrt(P)
    assert np.all(np.abs(res["grad"] - fd) < 4.5 * se + 1e-9), (res["grad"], fd, se)
    assert np.all(se < 0.1 * np.abs(fd))  # the check has power


def test_1d_sampler_quadrature_matches_fd_of_smoothed_objective():
    """E over the radial 1-D sampler of w (L(theta+tau) - L(theta-tau)) / 2, by generalised
    Gauss-Laguerre in x = -log(xi) (exact for a polynomial loss), equals the FD of L_sigma."""
    wl = _tiny_workload(1)
    target = oracle.render_target(wl)
    L = _loss_fn(wl, target)
    theta, sigma = float(wl.theta0[0]), float(wl.sigma[0])
    x, gw = roots_genlaguerre(40, 0.5)
    u = np.stack([np.exp(-x), np.full(x.size, 0.75)], 1)   # xi = e^-x, positive sign
    tau_t, w_t = oracle.sample_unit_batch(0, 1, u)
    tau, w = sigma * tau_t[:, 0], w_t[:, 0] / sigma
    diff = L(np.concatenate([theta + tau, theta - tau])[:, None])
    g_pair = 0.5 * w * (diff[: x.size] - diff[x.size:])
    # E_xi[g] = int_0^inf g(x) e^-x dx = int x^{1/2} (g(x) / x^{1/2}) e^-x dx
    expect_g = float((gw * g_pair / np.sqrt(x)).sum())
    fd = _fd5(lambda t: _smoothed_loss_gh(L, t, np.array([sigma]), n=40), np.array([theta]), 0)
    # agreement is limited only by the FP32 rounding of the rendered parameters
    assert expect_g == pytest.approx(fd, rel=2e-6)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    D = 7
    theta0 = rng.normal(size=D)
    grads = rng.normal(size=(25, D)) * np.logspace(-3, 1, D)
    p = torch.nn.Parameter(torch.tensor(theta0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=0.02, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = theta0.copy(), np.zeros(D), np.zeros(D)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        th, m, v = oracle.adam(th, m, v, g, t, 0.02)
        assert np.allclose(th, p.detach().numpy(), rtol=0, atol=1e-12)


def test_sigma_schedule():
    s0, smin, T = 0.125, 0.01, 300
    vals = [oracle.sigma_schedule(s0, smin, t, T) for t in range(T + 1)]
    assert all(v == s0 for v in vals[:150])
    assert vals[T] == pytest.approx(smin, abs=1e-15)
    assert vals[225] == pytest.approx(s0 - 0.5 * (s0 - smin), rel=1e-14)
    assert all(a >= b for a, b in zip(vals, vals[1:]))
