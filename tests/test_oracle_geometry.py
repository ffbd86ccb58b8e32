"""Pins of the oracle's geometric and boundary-data building blocks (CPU):
intersections against brute force, arc length against adaptive quadrature,
uniform sampling by surface measure, real spherical harmonics against scipy
and the identity printed for Example 3 (3D), harmonic-polynomial flux against
a finite-difference normal derivative."""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, special, stats

from paper_2508_16767_gb300 import workloads as wl


def star_problem(amp=0.15, k=5):
    a = [0.0] * (k + 1)
    b = [0.0] * (k + 1)
    a[k] = amp
    b[2] = 0.05
    return {"name": "star", "dim": 2,
            "surfaces": [{"kind": "star", "center": [0.1, -0.2], "radius": 1.0, "star_a": a, "star_b": b},
                         {"kind": "sphere", "center": [0.3, 0.1], "radius": 0.2}],
            "parent": [-1, 0], "sigma": [1.0, 3.0],
            "flux": [wl.fourier([0.3, -0.2], [0.5, 0.1], a0=0.0), wl.fourier([1.0, 0.5], [-0.3, 0.2])],
            "M": 3}


def star_xy(s, t):
    a, b = s["star_a"], s["star_b"]
    r = s["radius"] * (1 + sum(a[k] * np.cos(k * t) + b[k] * np.sin(k * t) for k in range(1, len(a))))
    return np.asarray(s["center"])[:, None] + np.stack([r * np.cos(t), r * np.sin(t)])


def brute_star_line(s, y, z, ray):
    """All intersections by a 400k-sample scan of the curve and Brent refinement."""
    t = np.linspace(0, 2 * np.pi, 400001)
    p = star_xy(s, t)
    f = (p[0] - y[0]) * z[1] - (p[1] - y[1]) * z[0]
    out = []
    for j in np.nonzero(np.signbit(f[:-1]) != np.signbit(f[1:]))[0]:
        g = lambda th: float((star_xy(s, np.array([th]))[0, 0] - y[0]) * z[1]
                             - (star_xy(s, np.array([th]))[1, 0] - y[1]) * z[0])
        th = optimize.brentq(g, t[j], t[j + 1], xtol=1e-15)
        q = star_xy(s, np.array([th]))[:, 0]
        tt = float(np.dot(q - y, z))
        if (tt > 1e-9) if ray else (abs(tt) > 1e-9):
            out.append(tt)
    return np.sort(out)


def test_star_intersections_match_brute_force(oracle_core):
    prob = star_problem(amp=0.3)
    s = prob["surfaces"][0]
    prep = oracle_core.Prepared(prob)
    rng = np.random.default_rng(0)
    n_multi = 0
    for trial in range(100):
        z = rng.standard_normal(2)
        z /= np.linalg.norm(z)
        if trial % 2 == 0:        # line through a point of the curve
            th = rng.uniform(0, 2 * np.pi)
            y = star_xy(s, np.array([th]))[:, 0]
            ray = False
        else:                     # ray from an interior point
            y = np.asarray(s["center"]) + rng.uniform(-0.5, 0.5, 2)
            ray = True
        ts = oracle_core.intersections(prob, 0, y, z, ray, prepared=prep)
        ref = brute_star_line(s, y, z, ray)
        assert len(ts) == len(ref)
        assert np.allclose(ts, ref, atol=1e-10)
        n_multi += len(ts) > 1
    assert n_multi > 5   # the star is non-convex: several crossings occur


def test_star_near_tangent_lines(oracle_core):
    """Lines through a curve point at a small angle to the tangent: the second
    crossing can lie within one scan step of the start point and must be found."""
    prob = star_problem(amp=0.3)
    s = prob["surfaces"][0]
    prep = oracle_core.Prepared(prob)
    found_close = 0
    for th in np.linspace(0.05, 2 * np.pi, 37):
        p0 = star_xy(s, np.array([th]))[:, 0]
        tan = star_xy(s, np.array([th + 1e-7]))[:, 0] - star_xy(s, np.array([th - 1e-7]))[:, 0]
        tan /= np.linalg.norm(tan)
        for ang in (3e-3, 1e-3, -1e-3, 3e-4):
            c, sn = np.cos(ang), np.sin(ang)
            z = np.array([c * tan[0] - sn * tan[1], sn * tan[0] + c * tan[1]])
            ts = oracle_core.intersections(prob, 0, p0, z, False, prepared=prep)
            ref = brute_star_line(s, p0, z, False)
            assert len(ts) == len(ref), (th, ang, ts, ref)
            assert np.allclose(ts, ref, atol=1e-9)
            found_close += int(np.any(np.abs(ref) < 2 * np.pi / 4096))
    assert found_close > 0


def test_sphere_intersections(oracle_core):
    for d in [2, 3, 6]:
        prob = {"dim": d, "surfaces": [{"kind": "sphere", "center": [0.1] * d, "radius": 0.7}],
                "parent": [-1], "sigma": [1.0], "flux": [wl.zero_flux()], "M": 1}
        rng = np.random.default_rng(d)
        c = np.full(d, 0.1)
        for _ in range(20):
            z = rng.standard_normal(d); z /= np.linalg.norm(z)
            u = rng.standard_normal(d); u /= np.linalg.norm(u)
            y = c + 0.7 * u                            # on the sphere: the line hits once more
            ts = oracle_core.intersections(prob, 0, y, z, False)
            assert len(ts) == 1
            assert abs(np.linalg.norm(y + ts[0] * z - c) - 0.7) < 1e-12
            assert abs(ts[0] + 2 * np.dot(z, y - c)) < 1e-12
            y2 = c + 0.3 * u                           # inside: the ray exits once
            ts = oracle_core.intersections(prob, 0, y2, z, True)
            assert len(ts) == 1 and ts[0] > 0
            assert abs(np.linalg.norm(y2 + ts[0] * z - c) - 0.7) < 1e-12


def test_star_arclength_matches_quadrature(oracle_core):
    prob = star_problem()
    s = prob["surfaces"][0]
    prep = oracle_core.Prepared(prob)
    speed = lambda t: np.linalg.norm(np.gradient(star_xy(s, np.array([t - 1e-6, t, t + 1e-6])), 1e-6, axis=1)[:, 1])
    for t in [0.3, 1.7, 3.1, 4.9, 2 * np.pi]:
        ref, _ = integrate.quad(speed, 0, t, epsabs=1e-12, limit=400)
        assert abs(oracle_core.star_arclen(prob, 0, t, prepared=prep) - ref) < 1e-7
    assert abs(prep.area[0] - oracle_core.star_arclen(prob, 0, 2 * np.pi, prepared=prep)) < 1e-12


def test_uniform_on_star_by_arclength(oracle_core):
    """Eq. naive_woi_p0: y_0 uniform by surface measure; the arc-length
    coordinate of the samples is U(0, L) (KS test)."""
    prob = star_problem()
    prep = oracle_core.Prepared(prob)
    y = oracle_core.uniform_points(prob, 0, 4000, seed=5, prepared=prep)
    c = np.asarray(prob["surfaces"][0]["center"])
    th = np.mod(np.arctan2(y[:, 1] - c[1], y[:, 0] - c[0]), 2 * np.pi)
    s = np.array([oracle_core.star_arclen(prob, 0, t, prepared=prep) for t in th]) / prep.area[0]
    assert stats.kstest(s, "uniform").pvalue > 1e-3
    # the samples lie on the curve
    assert np.allclose(star_xy(prob["surfaces"][0], th).T, y, atol=1e-12)


@pytest.mark.parametrize("d", [3, 6])
def test_uniform_on_sphere(oracle_core, d):
    prob = {"dim": d, "surfaces": [{"kind": "sphere", "center": [0.2] * d, "radius": 0.5}],
            "parent": [-1], "sigma": [1.0], "flux": [wl.zero_flux()], "M": 1}
    y = oracle_core.uniform_points(prob, 0, 5000, seed=3)
    u = (y - 0.2) / 0.5
    assert np.allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-12)
    # the first coordinate of a uniform point on S^{d-1} has density ∝ (1-x^2)^{(d-3)/2}
    x = u[:, 0]
    cdf = lambda v: stats.beta.cdf((v + 1) / 2, (d - 1) / 2, (d - 1) / 2)
    assert stats.kstest(x, cdf).pvalue > 1e-3


def test_real_sh_against_scipy_and_example3(oracle_core):
    rng = np.random.default_rng(1)
    for _ in range(10):
        u = rng.standard_normal(3); u /= np.linalg.norm(u)
        polar = math.acos(u[2]); az = math.atan2(u[1], u[0])
        for l in range(0, 5):
            for m in range(-l, l + 1):
                Yc = special.sph_harm_y(l, abs(m), polar, az)  # complex, with the (-1)^m phase
                if m == 0:
                    ref = Yc.real
                elif m > 0:
                    ref = math.sqrt(2) * (-1) ** m * Yc.real
                else:
                    ref = math.sqrt(2) * (-1) ** m * Yc.imag
                assert abs(oracle_core.real_sh(l, m, u) - ref) < 1e-12
        # Example 3 (3D): sin(phi) cos(theta) = sqrt(4 pi / 3) Y_1^1
        assert abs(math.sin(polar) * math.cos(az) - math.sqrt(4 * math.pi / 3) * oracle_core.real_sh(1, 1, u)) < 1e-13


def test_harmonic_poly_flux_is_normal_derivative(oracle_core):
    rng = np.random.default_rng(4)
    for d in [2, 3]:
        terms = wl.random_harmonic_poly(d, rng)
        prob = {"dim": d, "surfaces": [{"kind": "sphere", "center": [0.1] * d, "radius": 0.8}],
                "parent": [-1], "sigma": [1.0], "flux": [wl.harmonic_poly(1.7, terms, d)], "M": 1}
        for _ in range(5):
            u = rng.standard_normal(d); u /= np.linalg.norm(u)
            y = 0.1 + 0.8 * u
            h = 1e-6
            fd = (wl.eval_poly(terms, y + h * u)[0] - wl.eval_poly(terms, y - h * u)[0]) / (2 * h)
            assert abs(oracle_core.flux_at(prob, 0, y) - 1.7 * fd[0]) < 1e-6


def test_vr_arcs(oracle_core):
    """Sec. 4.4: dOmega^+ = {beta >= 0}, dOmega^- = {beta < 0}; the arcs cover
    the surface and the uniform samples of each part carry the right sign."""
    prob = star_problem()
    prep = oracle_core.Prepared(prob, "vr")
    for h in range(2):
        assert abs(prep.part_len[h].sum() - prep.area[h]) < 1e-8
        for part in (0, 1):
            y = oracle_core.uniform_part_points(prob, h, part, 300, seed=7 + h, prepared=prep)
            beta = np.array([prep.beta_scale[h] * oracle_core.flux_at(prob, h, yy, prepared=prep) for yy in y])
            assert np.all(beta >= -1e-9) if part == 0 else np.all(beta < 1e-9)


@pytest.mark.parametrize("d", [3, 5])
def test_vr_hemispheres(oracle_core, d):
    """Sec. 4.4 in d >= 3: data linear in the unit vector, beta = a . u, has the
    hemispheres {a . u >= 0} and {a . u < 0} as parts, each of half the area.  The
    samples of each part lie on the sphere, carry the part's sign and are uniform
    there: E[a^ . u] = +/- Gamma(d/2) / (sqrt(pi) Gamma((d+1)/2)) (the mean of |u_1| on
    S^{d-1}), the orthogonal components average to 0 and E[u_k^2] = 1/d."""
    from math import gamma, pi, sqrt
    c = np.linspace(-0.1, 0.2, d)
    R = 0.8
    a = np.zeros(d)
    if d == 3:
        flux = wl.real_sh({(1, 1): 0.6, (1, 0): -0.8}, 1)            # Y_1^1 ~ x, Y_1^0 ~ z
        a[0], a[2] = 0.6, -0.8
    else:
        flux = wl.harmonic_poly(2.0, [(0.6, tuple(int(k == 1) for k in range(d))),
                                      (0.8, tuple(int(k == 3) for k in range(d))),
                                      (5.0, (0,) * d)], d)
        a[1], a[3] = 0.6, 0.8
    prob = {"dim": d, "surfaces": [wl._sphere(c, R)], "parent": [-1], "sigma": [1.0], "flux": [flux], "M": 1}
    prep = oracle_core.Prepared(prob, "vr")
    area = oracle_core.omega(d) * R ** (d - 1)
    assert prep.part_len[0] == pytest.approx([area / 2, area / 2], rel=1e-14)
    m1 = gamma(d / 2) / (sqrt(pi) * gamma((d + 1) / 2))
    n = 20000
    Q = np.linalg.qr(np.column_stack([a] + [np.eye(d)[k] for k in range(d)]))[0][:, 1:d]   # a^-perp basis
    for part, sgn in ((0, 1.0), (1, -1.0)):
        y = oracle_core.uniform_part_points(prob, 0, part, n, seed=3 + part, prepared=prep)
        u = (y - c) / R
        assert np.allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-13)
        beta = np.array([oracle_core.flux_at(prob, 0, yy, prepared=prep) for yy in y[:500]])
        assert np.all(sgn * beta >= 0)
        t = u @ a
        assert abs(t.mean() - sgn * m1) < 5 * t.std() / sqrt(n)
        p = u @ Q
        assert np.all(np.abs(p.mean(axis=0)) < 5 * p.std(axis=0) / sqrt(n))
        assert np.all(np.abs((u ** 2).mean(axis=0) - 1 / d) < 5 * (u ** 2).std(axis=0) / sqrt(n))


def test_vr_parts_in_3d(oracle_core):
    """Degree-2 data on a 3D sphere has no hemisphere parts, nor has any data on an
    ellipsoid: they are flagged for the start by uniform trials (-1)."""
    for prob in (wl.nested_3d_problem(), wl.ellipsoids_problem(3)):
        prep = oracle_core.Prepared(prob, "vr")
        assert np.all(prep.part_len < 0)
