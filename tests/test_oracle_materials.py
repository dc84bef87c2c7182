"""Pins of the oracle's smooth dielectric and of Russian roulette on the radiance.

The dielectric event (reflect with probability F, else refract) is checked against
the textbook optics it restates, in forms independent of the oracle's own:

* Fresnel amplitude ratios in their sine/tangent form (Hecht, Optics):
  r_s = -sin(i - t) / sin(i + t), r_p = tan(i - t) / tan(i + t), with the refraction
  angle t from Snell's law n_1 sin i = n_2 sin t; F = (r_s^2 + r_p^2) / 2;
* normal incidence: F = ((n - 1) / (n + 1))^2 = 0.04 for n = 1.5;
* Brewster's angle atan(n_2 / n_1): r_p = 0;
* total internal reflection beyond the critical angle asin(n_2 / n_1): F = 1;
* Stokes reciprocity: the same pair of angles reflects alike from either side;
* directions: the refracted ray is a unit vector in the plane of incidence obeying
  Snell's law, the reflected ray the mirror image; each new origin lies on the side
  its ray leaves into.

Russian roulette must leave the radiance unbiased: a path that survives with
probability q carries its throughput divided by q. In a white furnace a convex
diffuse object of albedo rho shows exactly rho on average with roulette at its first
vertex, and in a closed box the mean image with roulette equals the image without it.

Each pin is also run on copies of the oracle with a plausible mistake planted (a
dropped division by q, rs used for rp, eta not inverted, a wrong refraction term,
no total internal reflection, an origin on the wrong side): at least one check must
fail on every planted mistake.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import build as oracle_build
from workloads import MAT_DIELECTRIC, MAT_DIFFUSE, SceneBuilder, config_gi_box

N_GLASS = 1.5


def _ray(theta, phi=0.3):
    """Unit direction making angle theta with -z (hitting a surface of normal +z)."""
    return np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), -math.cos(theta)])


def _textbook(theta_i, n1, n2):
    """Fresnel amplitude ratios (sine/tangent form) and F for incidence theta_i."""
    theta_t = math.asin(n1 * math.sin(theta_i) / n2)
    rs = -math.sin(theta_i - theta_t) / math.sin(theta_i + theta_t)
    rp = math.tan(theta_i - theta_t) / math.tan(theta_i + theta_t)
    return rs, rp, 0.5 * (rs * rs + rp * rp), theta_t


# ----------------------------------------------------------------------------- checks
# Each check asserts one fact of optics about oracle.dielectric(); the tests below run
# them on the oracle, and on copies with planted mistakes.
def check_normal_incidence():
    up = np.array([0.0, 0.0, 1.0])
    out = oracle.dielectric([0, 0, -1.0], up, N_GLASS, 0.5)          # from outside
    inn = oracle.dielectric([0, 0, 1.0], up, N_GLASS, 0.5)           # from inside the glass
    f0 = ((N_GLASS - 1) / (N_GLASS + 1)) ** 2
    assert abs(out["F"] - f0) < 1e-15 and abs(inn["F"] - f0) < 1e-15, (out["F"], inn["F"], f0)
    assert abs(f0 - 0.04) < 1e-15


def check_textbook_fresnel():
    up = np.array([0.0, 0.0, 1.0])
    for deg in np.linspace(0.5, 89.5, 179):
        i = math.radians(deg)
        rs, rp, F, _ = _textbook(i, 1.0, N_GLASS)  # from outside
        r = oracle.dielectric(_ray(i), up, N_GLASS, 0.5)
        assert abs(r["F"] - F) < 1e-12 and abs(r["rs"] - rs) < 1e-12 and abs(r["rp"] - rp) < 1e-12, (deg, r, F)
    crit = math.asin(1.0 / N_GLASS)
    for deg in np.linspace(0.5, math.degrees(crit) - 0.5, 80):
        i = math.radians(deg)
        rs, rp, F, _ = _textbook(i, N_GLASS, 1.0)  # from inside: the ray leaves along +z
        r = oracle.dielectric(-_ray(i), up, N_GLASS, 0.5)
        assert abs(r["F"] - F) < 1e-11 and abs(r["rs"] - rs) < 1e-11 and abs(r["rp"] - rp) < 1e-11, (deg, r, F)


def check_brewster():
    up = np.array([0.0, 0.0, 1.0])
    for n1, n2, sgn in ((1.0, N_GLASS, 1.0), (N_GLASS, 1.0, -1.0)):
        ib = math.atan(n2 / n1)
        r = oracle.dielectric(sgn * _ray(ib), up, N_GLASS, 0.5)
        assert abs(r["rp"]) < 1e-14, (n1, r)
        assert abs(r["F"] - 0.5 * r["rs"] ** 2) < 1e-15
        # at Brewster's angle i + t = 90 degrees, so r_s = -sin(i - t) = cos(2 i)
        assert abs(r["rs"] - math.cos(2 * ib)) < 1e-14, (r["rs"], math.cos(2 * ib))


def check_total_internal_reflection():
    up = np.array([0.0, 0.0, 1.0])
    crit = math.asin(1.0 / N_GLASS)
    for deg in (math.degrees(crit) + 0.01, 50.0, 70.0, 89.0):
        d = -_ray(math.radians(deg))  # inside the glass, heading out
        r = oracle.dielectric(d, up, N_GLASS, 1.0 - 2.0 ** -24)  # the largest uniform still reflects
        assert r["F"] == 1.0 and r["reflected"], (deg, r)
        mirror = d - 2.0 * np.dot(d, up) * up
        assert np.allclose(r["dir"], mirror, atol=1e-14)
        assert r["org"][2] < 0.0  # stays inside
    below = oracle.dielectric(-_ray(crit - 1e-3), up, N_GLASS, 0.999)
    assert below["F"] < 1.0 and not below["reflected"]


def check_stokes_reciprocity():
    up = np.array([0.0, 0.0, 1.0])
    for deg in np.linspace(1.0, 89.0, 45):
        i = math.radians(deg)
        t = math.asin(math.sin(i) / N_GLASS)
        a = oracle.dielectric(_ray(i), up, N_GLASS, 0.5)["F"]
        b = oracle.dielectric(-_ray(t), up, N_GLASS, 0.5)["F"]
        assert abs(a - b) < 1e-12, (deg, a, b)


def check_directions():
    rng = np.random.default_rng(17)
    for _ in range(400):
        ng = rng.normal(size=3)
        ng /= np.linalg.norm(ng)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if abs(np.dot(d, ng)) < 1e-3:
            continue
        p = rng.normal(size=3)
        outside = np.dot(d, ng) < 0.0
        n1, n2 = (1.0, N_GLASS) if outside else (N_GLASS, 1.0)
        n_inc = ng if outside else -ng            # normal on the incident side
        sin_i = np.linalg.norm(np.cross(d, n_inc))
        refr = oracle.dielectric(d, ng, N_GLASS, 1.0 - 2.0 ** -24, p)
        refl = oracle.dielectric(d, ng, N_GLASS, 2.0 ** -24, p)
        # reflection: the mirror image, leaving on the incident side
        assert refl["reflected"]
        assert np.allclose(refl["dir"], d - 2.0 * np.dot(d, ng) * ng, atol=1e-12)
        assert np.dot(refl["org"] - p, n_inc) > 0.0 and abs(np.linalg.norm(refl["org"] - p) - 1e-4) < 1e-12
        if n1 * sin_i >= n2:  # total internal reflection: every u reflects
            assert refr["reflected"] and refr["F"] == 1.0
            continue
        t = refr["dir"]
        assert not refr["reflected"]
        assert abs(np.linalg.norm(t) - 1.0) < 1e-12
        assert abs(n1 * sin_i - n2 * np.linalg.norm(np.cross(t, n_inc))) < 1e-12       # Snell
        assert abs(np.dot(t, np.cross(d, n_inc))) < 1e-12                               # plane of incidence
        assert np.dot(t, n_inc) < 0.0                                                    # crosses the surface
        assert np.dot(np.cross(n_inc, t), np.cross(n_inc, d)) > 0.0                     # same side of the normal
        assert np.dot(refr["org"] - p, n_inc) < 0.0 and abs(np.linalg.norm(refr["org"] - p) - 1e-4) < 1e-12


def _furnace_scene(albedo):
    b = SceneBuilder()
    m = b.material(MAT_DIFFUSE, albedo)
    b.sphere((0, 0, 0), 1.0, m)
    b.look_at((0, -5, 0), (0, 0, 0), (0, 0, 1), 30.0)
    b.background[:] = 1.0
    return b.build()


def check_roulette_furnace():
    """Convex diffuse sphere under a uniform environment of radiance 1, roulette from the
    first vertex: each sample through the sphere is 0 (killed) or albedo / q (q = min(0.95,
    max albedo)), whose mean is the albedo. The mean over the sphere's pixels must equal the
    albedo within 4.5 standard errors, per channel."""
    for albedo in ((0.5, 0.5, 0.5), (0.9, 0.3, 0.6)):
        sc = _furnace_scene(albedo)
        W = H = 40
        S = 32
        img = oracle.render(sc, np.array([[2, 0, 0]], np.int32), np.array([[albedo[0]]], np.float32), W, H, S,
                            depth=3, rr_start=0, seed=5)[0]
        # pixels whose every sample meets the sphere (the central disk)
        y, x = np.mgrid[0:H, 0:W]
        r_pix = math.atan(1.0 / math.sqrt(24.0)) / math.tan(math.radians(15.0)) * (W / 2)
        inner = (x + 0.5 - W / 2) ** 2 + (y + 0.5 - H / 2) ** 2 < (r_pix - 2.0) ** 2
        rho = np.asarray(albedo, np.float32).astype(np.float64)
        q = min(0.95, rho.max())
        vals = img[inner]                                # [m, 3] pixel means over S samples
        # every sample is 0 or rho / q: a pixel mean is k / S times rho / q
        k = vals / (rho / q) * S
        assert np.all(np.abs(k - np.round(k)) < 1e-9), "a sample is neither 0 nor albedo / q"
        mean = vals.mean(axis=0)
        se = np.sqrt(q * (1 - q)) * (rho / q) / math.sqrt(vals.shape[0] * S)
        assert np.all(np.abs(mean - rho) <= 4.5 * se), (albedo, mean, rho, se)


def check_roulette_unbiased_in_closed_box():
    """The GI box (diffuse walls, boxes, a mirror sphere, a ceiling light) at depth 6: the
    mean image with roulette from vertex 1 equals the image without roulette within 4.5
    standard errors of the per-pixel difference (pixels are independent paths)."""
    wl = config_gi_box()
    W = H = 32
    S = 16
    th = wl.theta_ref[None]
    a = oracle.render(wl.scene, wl.bindings, th, W, H, S, depth=6, rr_start=-1, seed=9)[0]
    b = oracle.render(wl.scene, wl.bindings, th, W, H, S, depth=6, rr_start=1, seed=9)[0]
    d = (b - a).reshape(-1, 3).sum(axis=1)
    se = d.std(ddof=1) / math.sqrt(d.size)
    assert abs(d.mean()) <= 4.5 * se, (d.mean(), se)
    assert not np.allclose(a, b)  # roulette changed individual paths


PINS = [check_normal_incidence, check_textbook_fresnel, check_brewster, check_total_internal_reflection,
        check_stokes_reciprocity, check_directions, check_roulette_furnace, check_roulette_unbiased_in_closed_box]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


# ----------------------------------------------------------------------------- planted mistakes
MISTAKES = {
    "roulette_without_division": {"beta = mul(beta, 1.0 / q);": ""},
    "rp_equals_rs": {"double rp = (ci - eta * ct) / (ci + eta * ct);": "double rp = (eta * ci - ct) / (eta * ci + ct);"},
    "eta_not_inverted": {"if (ci > 0.0) { eta = 1.0 / ior; n = ng; }": "if (ci > 0.0) { eta = ior; n = ng; }"},
    "refraction_term_sign": {"mul(n, eta * ci - ct)": "mul(n, eta * ci + ct)"},
    "no_total_internal_reflection": {"if (s2t >= 1.0) {": "if (s2t >= 1.0e30) {"},
    "refracted_origin_on_incident_side": {"*org_out = sub(p, mul(n, ORC_EPS));": "*org_out = add(p, mul(n, ORC_EPS));"},
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_a_pin_fails_on_a_planted_mistake(name, tmp_path):
    path = oracle_build.build_modified(MISTAKES[name], str(tmp_path))
    failed = []
    with oracle.library(path):
        for pin in PINS:
            try:
                with np.errstate(all="ignore"):
                    pin()
            except AssertionError:
                failed.append(pin.__name__)
    assert failed, f"no pin fails with the planted mistake {name}"
