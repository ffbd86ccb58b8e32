"""Pins of the oracle's ellipsoid surfaces and point-charge data (CPU), the
geometry of the paper's Example 2 (Sec. 5):

* the area of an ellipsoid against the closed forms of spheroids and spheres and
  against a direct two-dimensional quadrature of the area element (triaxial);
* line / ray intersections against brute-force root finding along the line;
* uniform sampling by surface measure: the divergence-theorem identities
  int n dA = 0 and int (y - c).n dA = d |E|, which the sphere-mapped density
  (no rejection) violates by many standard errors on the same ellipsoid;
* an ellipsoid with A = I / R^2 walks exactly like the sphere of radius R;
* the point-charge flux against a finite-difference normal derivative;
* the Example 2 workload: the estimate equals the manufactured solution
  |x|^{2-d} up to one additive constant.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

from paper_2508_16767_gb300 import workloads as wl


def one_ellipsoid(d, A, c=None, flux=None):
    c = np.zeros(d) if c is None else np.asarray(c, dtype=np.float64)
    return {"dim": d, "surfaces": [wl._ellipsoid(c, A)], "parent": [-1], "sigma": [1.0],
            "flux": [flux or wl.zero_flux()], "M": 1}


def rotated(diag_lam, seed):
    d = len(diag_lam)
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((d, d)))
    return Q @ np.diag(diag_lam) @ Q.T


def test_area_closed_forms_and_quadrature(oracle_core):
    # spheres
    for d in (3, 4, 6):
        R = 0.7
        assert oracle_core.ellipsoid_area(d, np.full(d, 1 / R ** 2)) == pytest.approx(
            oracle_core.omega(d) * R ** (d - 1), rel=1e-12)
    # oblate and prolate spheroids
    a, c = 1.0, 0.5
    e = math.sqrt(1 - c * c / (a * a))
    S = 2 * math.pi * a * a * (1 + (1 - e * e) / e * math.atanh(e))
    assert oracle_core.ellipsoid_area(3, np.array([1 / a ** 2, 1 / a ** 2, 1 / c ** 2])) == pytest.approx(S, rel=1e-12)
    a, c = 0.5, 1.5
    e = math.sqrt(1 - a * a / (c * c))
    S = 2 * math.pi * a * a * (1 + c / (a * e) * math.asin(e))
    assert oracle_core.ellipsoid_area(3, np.array([1 / a ** 2, 1 / a ** 2, 1 / c ** 2])) == pytest.approx(S, rel=1e-12)
    # triaxial: |F_theta x F_phi| of F = diag(a) (sin th cos ph, sin th sin ph, cos th)
    ax = np.array([1.0, 0.6, 0.35])

    def elem(ph, th):
        Ft = ax * np.array([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
        Fp = ax * np.array([-np.sin(th) * np.sin(ph), np.sin(th) * np.cos(ph), 0.0])
        return np.linalg.norm(np.cross(Ft, Fp))

    ref, _ = integrate.dblquad(elem, 0, math.pi, 0, 2 * math.pi, epsabs=1e-12, epsrel=1e-12)
    assert oracle_core.ellipsoid_area(3, ax ** -2.0) == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("d", [3, 5])
def test_ellipsoid_intersections(oracle_core, d):
    A = rotated(np.linspace(1.0, 9.0, d), 11 + d)
    c = np.linspace(-0.2, 0.3, d)
    prob = one_ellipsoid(d, A, c)
    prep = oracle_core.Prepared(prob)
    lam, R = np.linalg.eigh(A)
    rng = np.random.default_rng(d)
    form = lambda p: float((p - c) @ A @ (p - c))
    for _ in range(25):
        z = rng.standard_normal(d); z /= np.linalg.norm(z)
        u = rng.standard_normal(d); u /= np.linalg.norm(u)
        y = c + R @ (u / np.sqrt(lam))                   # on the surface
        ts = oracle_core.intersections(prob, 0, y, z, False, prepared=prep)
        # brute force: sign changes of the form along the line, then Brent
        grid = np.linspace(-4, 4, 8001)
        f = np.array([form(y + t * z) - 1 for t in grid])
        brute = [optimize.brentq(lambda t: form(y + t * z) - 1, grid[j], grid[j + 1], xtol=1e-15)
                 for j in np.nonzero(np.signbit(f[:-1]) != np.signbit(f[1:]))[0]]
        brute = [t for t in brute if abs(t) > 1e-9]
        assert len(ts) == 1 == len(brute)
        assert abs(ts[0] - brute[0]) < 1e-10
        assert abs(form(y + ts[0] * z) - 1) < 1e-11
        y2 = c + R @ (0.4 * u / np.sqrt(lam))            # inside: the ray exits once
        ts = oracle_core.intersections(prob, 0, y2, z, True, prepared=prep)
        assert len(ts) == 1 and ts[0] > 0 and abs(form(y2 + ts[0] * z) - 1) < 1e-11


def test_uniform_on_ellipsoid_by_area(oracle_core):
    """Eq. naive_woi_p0 on an ellipsoid: the samples lie on the surface and satisfy
    int n dA = 0 and |dE| E[(y - c).n] = d |E| (divergence theorem); the
    sphere-mapped density (no rejection) misses the second by many SE."""
    d = 3
    A = rotated([1.0, 4.0, 16.0], 5)
    c = np.array([0.1, -0.2, 0.05])
    prob = one_ellipsoid(d, A, c)
    prep = oracle_core.Prepared(prob)
    y = oracle_core.uniform_points(prob, 0, 20000, seed=9, prepared=prep)
    e = y - c
    assert np.allclose(np.einsum("ni,ij,nj->n", e, A, e), 1.0, atol=1e-12)
    g = e @ A
    n = g / np.linalg.norm(g, axis=1)[:, None]
    vol = (4 * math.pi / 3) / math.sqrt(np.linalg.det(A))
    area = prep.area[0]
    se = lambda v: v.std() / math.sqrt(len(v))
    for k in range(d):
        assert abs(n[:, k].mean()) < 5 * se(n[:, k])
    s = np.einsum("ni,ni->n", e, n)
    assert abs(area * s.mean() - d * vol) < 5 * area * se(s)
    # the mapped density without rejection: the same statistic is far off
    lam, R = np.linalg.eigh(A)
    u = np.random.default_rng(1).standard_normal((20000, d))
    u /= np.linalg.norm(u, axis=1)[:, None]
    em = (u / np.sqrt(lam)) @ R.T
    gm = em @ A
    sm = np.einsum("ni,ni->n", em, gm / np.linalg.norm(gm, axis=1)[:, None])
    assert abs(area * sm.mean() - d * vol) > 20 * area * se(sm)


def sphere_pair(d, as_ellipsoid):
    c0 = np.zeros(d)
    c1 = np.zeros(d)
    c1[0], c1[1] = 0.2, -0.1
    R0, R1 = 1.0, 0.45
    ex = tuple(1 if k == 0 else 0 for k in range(d))
    ey = tuple(1 if k == 1 else 0 for k in range(d))

    def surf(c, R):
        return wl._ellipsoid(c, np.eye(d) / R ** 2) if as_ellipsoid else wl._sphere(c, R)

    x0 = np.zeros(d)
    x0[0] = 3.0
    return {"dim": d, "surfaces": [surf(c0, R0), surf(c1, R1)], "parent": [-1, 0], "sigma": [1.0, 3.0],
            "flux": [wl.harmonic_poly(1.0, [(1.0, tuple(a + b for a, b in zip(ex, ey)))], d),
                     {"basis": "point_charge", "coef": [0.7] + list(x0)}],
            "M": 6}


@pytest.mark.parametrize("d", [3, 5])
def test_sphere_as_ellipsoid_walks_identically(oracle_core, d):
    """A = I / R^2 accepts every first attempt, so the same Philox words give the
    same walk as on the sphere: per-walk tallies agree to rounding."""
    ps, pe = sphere_pair(d, False), sphere_pair(d, True)
    x = np.zeros(d)
    x[0], x[2] = -0.3, 0.25
    ids = np.arange(400, dtype=np.uint64)
    ws = oracle_core.walks(ps, x, ids, seed=3)
    we = oracle_core.walks(pe, x, ids, seed=3)
    assert np.array_equal(ws["H"], we["H"])
    assert np.all(np.abs(ws["u"] - we["u"]) <= 1e-12 * ws["scale"][:, 0])
    assert np.all(np.abs(ws["grad"] - we["grad"]).max(axis=1) <= 1e-12 * ws["scale"][:, 1])


def test_point_charge_flux_is_normal_derivative(oracle_core):
    d = 4
    A = rotated([1.0, 2.0, 3.0, 5.0], 2)
    c = np.array([1.4, 0.0, 0.1, 0.0])
    x0 = np.array([-0.2, 0.1, 0.0, 0.3])
    prob = one_ellipsoid(d, A, c, {"basis": "point_charge", "coef": [1.7] + list(x0)})
    prep = oracle_core.Prepared(prob)
    lam, R = np.linalg.eigh(A)
    rng = np.random.default_rng(4)
    u_pc = lambda p: np.linalg.norm(p - x0) ** (2 - d)
    for _ in range(10):
        u = rng.standard_normal(d); u /= np.linalg.norm(u)
        y = c + R @ (u / np.sqrt(lam))
        g = A @ (y - c)
        n = g / np.linalg.norm(g)
        h = 1e-5
        fd = (u_pc(y + h * n) - u_pc(y - h * n)) / (2 * h)
        assert oracle_core.flux_at(prob, 0, y, prepared=prep) == pytest.approx(1.7 * fd, rel=1e-7)


def test_example2_matches_point_charge_up_to_a_constant(oracle_core):
    """3D nested ellipsoids of Example 2 with the point-charge data (M = 5, as in
    the paper's table): the estimate is the single-layer representation, equal
    to |x|^{-1} up to one additive constant (Sec. 1).  After removing the
    SE-weighted mean offset, every point agrees within 4 SE plus a truncation
    allowance of 0.02 (the paper's relative error at M = 5 levels off near 1.2 %).
    The conductivity ratios of this workload are close to 1, so the interface
    jumps move u by less than this band: the test pins the outer data and the
    ellipsoid transitions; the jump terms are pinned by the sphere identity
    above and by the sphere closed forms."""
    prob = wl.ellipsoids_problem(3)
    x = wl.ellipsoid_points(prob, 8, seed=21)
    est = oracle_core.estimate(prob, x, 1_000_000, seed=1, M=5)
    u, _ = wl.point_charge(x)
    off = est["u"] - u
    w = 1.0 / est["se_u"] ** 2
    shift = float(np.sum(w * off) / np.sum(w))
    assert np.all(np.abs(off - shift) <= 4 * est["se_u"] + 0.02), (off - shift, est["se_u"])
