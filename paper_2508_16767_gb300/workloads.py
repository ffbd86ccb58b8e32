"""Seeded synthetic inputs for the Walk-on-Interfaces estimator.

This module only builds problem descriptions (geometry, conductivities,
boundary/interface flux data) and evaluation points.  It holds none of the
estimator's arithmetic: no alpha/beta scaling, no schedule, no sampling.  The
CUDA library and the CPU oracle both consume what it returns, each converting
it with its own code.

Problem dictionary (JSON-compatible):

    dim       int, 2..6
    surfaces  list of {"kind": "sphere" | "star" | "ellipsoid" | "mesh", "center": [dim],
              "radius": R, "star_a": [K+1], "star_b": [K+1], "matrix": [dim][dim],
              "vertices": [nv][3], "triangles": [nt][3]}
              (star: 2D only, r(t) = R (1 + sum_k a_k cos kt + b_k sin kt), index 0
              unused; ellipsoid: d >= 3, (y - c)^T A (y - c) = 1 with A = matrix
              symmetric positive definite; mesh: 3D, closed, triangles counter-
              clockwise seen from outside, "center" any reference point inside)
    parent    list of int, parent[0] = -1 (the outer boundary dOmega_1),
              parent[i] = index of the region that contains region i
    sigma     list of float, conductivity inside each region (sigma_1 > 0)
    flux      list of {"basis": ..., "coef": [...]}:
              "zero"           b = 0
              "fourier"        [a0, a1, b1, ..., aK, bK] in the local parameter
                               angle of a 2D circle or star
              "real_sh"        coef[l*l + l + m], orthonormal real spherical
                               harmonics of the unit direction from the centre (3D)
              "harmonic_poly"  [s, T, (c, e_1..e_dim) x T]: b(y) = s n(y).grad P(y)
                               with P(y) = sum c prod y_k^e_k harmonic
              "point_charge"   [s, x0_1..x0_dim]: b(y) = s n(y).grad |y - x0|^{2-dim}
                               (dim >= 3)
    M         default truncation for this workload

The recipes follow the synthetic workloads used to measure the estimator:
nested layers (2D, 3D, 6D), a star-shaped domain with many small inclusions,
and a batch of heterogeneous manufactured-solution instances.
"""
from __future__ import annotations

import math

import numpy as np


def _sphere(center, radius):
    return {"kind": "sphere", "center": [float(c) for c in center], "radius": float(radius)}


def _ellipsoid(center, matrix):
    return {"kind": "ellipsoid", "center": [float(c) for c in center],
            "matrix": [[float(v) for v in row] for row in np.asarray(matrix, dtype=np.float64)]}


def _star(center, radius, a, b):
    return {"kind": "star", "center": [float(c) for c in center], "radius": float(radius),
            "star_a": [float(v) for v in a], "star_b": [float(v) for v in b]}


def fourier(coefs_cos, coefs_sin, a0=0.0):
    """[a0, a1, b1, ..., aK, bK] from cos / sin coefficient lists (k = 1..K)."""
    out = [float(a0)]
    for a, b in zip(coefs_cos, coefs_sin):
        out += [float(a), float(b)]
    return {"basis": "fourier", "coef": out}


def real_sh(coef_by_lm, lmax):
    """coef[l*l + l + m] from a {(l, m): value} dict."""
    out = [0.0] * ((lmax + 1) ** 2)
    for (l, m), v in coef_by_lm.items():
        out[l * l + l + m] = float(v)
    return {"basis": "real_sh", "coef": out}


def harmonic_poly(scale, terms, dim):
    """b = scale * n . grad P with P = sum c * prod y_k^e_k; terms = [(c, (e_1..e_d)), ...]."""
    out = [float(scale), float(len(terms))]
    for c, e in terms:
        assert len(e) == dim
        out += [float(c)] + [float(v) for v in e]
    return {"basis": "harmonic_poly", "coef": out}


def zero_flux():
    return {"basis": "zero", "coef": []}


# ---------------------------------------------------------------------------
# layered workloads
# ---------------------------------------------------------------------------

def concentric_2d_problem():
    """Unit disk with a concentric inclusion r = 0.5, sigma = (1, 2), Neumann
    flux cos(theta) on |x| = 1 and flux jump 0.5 cos(theta) on r = 0.5."""
    return {
        "name": "2d-concentric", "dim": 2,
        "surfaces": [_sphere([0, 0], 1.0), _sphere([0, 0], 0.5)],
        "parent": [-1, 0], "sigma": [1.0, 2.0],
        "flux": [fourier([1.0], [0.0]), fourier([0.5], [0.0])],
        "M": 4,
    }


def concentric_2d_points():
    """64 points on a polar grid: r_k = (2k+1)/16, theta_j = pi/8 + j pi/4."""
    pts = []
    for k in range(8):
        r = (2 * k + 1) / 16.0
        for j in range(8):
            t = math.pi / 8 + j * math.pi / 4
            pts.append([r * math.cos(t), r * math.sin(t)])
    return np.asarray(pts, dtype=np.float64)


def nested_3d_problem(seed=2):
    """Spheres r = 1, 0.8, 0.5 nested, sigma = (1, 5, 0.2); Neumann flux
    Y_1^0 + 0.3 Y_2^1; flux jumps sum_m a_m Y_2^m with a ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    a2 = rng.standard_normal(5)
    a3 = rng.standard_normal(5)
    return {
        "name": "3d-nested", "dim": 3,
        "surfaces": [_sphere([0, 0, 0], 1.0), _sphere([0, 0, 0], 0.8), _sphere([0, 0, 0], 0.5)],
        "parent": [-1, 0, 1], "sigma": [1.0, 5.0, 0.2],
        "flux": [real_sh({(1, 0): 1.0, (2, 1): 0.3}, 2),
                 real_sh({(2, m): a2[m + 2] for m in range(-2, 3)}, 2),
                 real_sh({(2, m): a3[m + 2] for m in range(-2, 3)}, 2)],
        "M": 6,
    }


def linear_3d_problem():
    """Concentric spheres r = 1, 0.7, 0.4, sigma = (1, 3, 0.5) with data linear in the
    unit vector: Neumann flux Y_1^0 + 0.4 Y_1^{-1}, no jump on r = 0.7, and the jump
    0.5 n . grad(x_1 + 0.6 x_3 + 2) on r = 0.4 (the constant term has no gradient).
    Every sign part is a hemisphere, the case of the variance-reduced walk in 3D."""
    return {
        "name": "3d-linear", "dim": 3,
        "surfaces": [_sphere([0, 0, 0], 1.0), _sphere([0, 0, 0], 0.7), _sphere([0, 0, 0], 0.4)],
        "parent": [-1, 0, 1], "sigma": [1.0, 3.0, 0.5],
        "flux": [real_sh({(1, 0): 1.0, (1, -1): 0.4}, 1), zero_flux(),
                 harmonic_poly(0.5, [(1.0, (1, 0, 0)), (0.6, (0, 0, 1)), (2.0, (0, 0, 0))], 3)],
        "M": 6,
    }


def zonal_3d_problem():
    """Concentric spheres r = 1, 0.5, sigma = (1, 4) with degree-2 data Y_2^0 on the outer
    sphere and the jump -0.5 Y_2^0 + 0.3 Y_2^2 on the inner one.  The sign parts are not
    halves (Y_2^0 >= 0 on 1 - 1/sqrt(3) of the sphere) and have no closed form in general:
    the case of the variance-reduced start by uniform trials."""
    return {
        "name": "3d-zonal", "dim": 3,
        "surfaces": [_sphere([0, 0, 0], 1.0), _sphere([0, 0, 0], 0.5)],
        "parent": [-1, 0], "sigma": [1.0, 4.0],
        "flux": [real_sh({(2, 0): 1.0}, 2), real_sh({(2, 0): -0.5, (2, 2): 0.3}, 2)],
        "M": 6,
    }


def ball_points(n, dim, seed, radius=1.0):
    """n points uniform in the ball of the given radius (r = R U^{1/d})."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, dim))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / dim)
    return g * r[:, None]


def nested_nd_problem(dim, M=8):
    """Hyperspheres r = 1, 0.6 in d dimensions (3 <= d <= 6), sigma = (1, 4); Neumann
    flux x_1 on |x| = 1 and flux jump x_2 on the inner sphere (0.6 x_2/|x| there)."""
    d = dim
    e1 = tuple(1 if k == 0 else 0 for k in range(d))
    e2 = tuple(1 if k == 1 else 0 for k in range(d))
    return {
        "name": f"{d}d-nested", "dim": d,
        "surfaces": [_sphere([0] * d, 1.0), _sphere([0] * d, 0.6)],
        "parent": [-1, 0], "sigma": [1.0, 4.0],
        "flux": [harmonic_poly(1.0, [(1.0, e1)], d), harmonic_poly(0.6, [(1.0, e2)], d)],
        "M": M,
    }


def nested_6d_problem():
    """The 6D workload: nested_nd_problem in six dimensions, M = 8."""
    return nested_nd_problem(6)


# ---------------------------------------------------------------------------
# star-shaped domain with many inclusions
# ---------------------------------------------------------------------------

def _star_radius(a, b, t):
    s = np.ones_like(t)
    for k in range(1, len(a)):
        s = s + a[k] * np.cos(k * t) + b[k] * np.sin(k * t)
    return s


def _star_curve(a, b, n=4096):
    t = np.linspace(0.0, 2 * np.pi, n, endpoint=False)
    r = _star_radius(a, b, t)
    return t, np.stack([r * np.cos(t), r * np.sin(t)], axis=1)


def _inside_star(a, b, p):
    t = np.arctan2(p[..., 1], p[..., 0])
    return np.linalg.norm(p, axis=-1) < _star_radius(a, b, t)


def star_inclusions_problem(seed=3, n_incl=32, star_amp=0.15, star_k=5):
    """Star r(t) = 1 + 0.15 cos 5t with 32 circles (radii U[0.03, 0.08], a
    gap >= 0.02 to each other and to the star), sigma_1 = 1, sigma_i
    log-uniform on [0.1, 10]; flux jumps are random trig polynomials of degree
    <= 4 with N(0,1) coefficients in the local angle (zero mean); the Neumann
    flux is the same in the global angle minus its arc-length mean."""
    rng = np.random.default_rng(seed)
    a = [0.0] * (star_k + 1)
    b = [0.0] * (star_k + 1)
    a[star_k] = star_amp
    _, curve = _star_curve(a, b)
    circles = []
    tries = 0
    while len(circles) < n_incl and tries < 200000:
        tries += 1
        rad = rng.uniform(0.03, 0.08)
        c = rng.uniform(-1.2, 1.2, size=2)
        if not _inside_star(a, b, c):
            continue
        if np.min(np.linalg.norm(curve - c, axis=1)) < rad + 0.02:
            continue
        if any(np.linalg.norm(c - c2) < rad + r2 + 0.02 for c2, r2 in circles):
            continue
        circles.append((c, rad))
    surfaces = [_star([0, 0], 1.0, a, b)] + [_sphere(c, r) for c, r in circles]
    n = len(surfaces)
    sigma = [1.0] + list(np.exp(rng.uniform(math.log(0.1), math.log(10.0), n - 1)))
    flux = []
    # Neumann flux in the global angle, projected to zero arc-length mean
    ca, cb = rng.standard_normal(4), rng.standard_normal(4)
    t = np.linspace(0.0, 2 * np.pi, 8192, endpoint=False)
    r = _star_radius(a, b, t)
    dr = sum(-k * a[k] * np.sin(k * t) + k * b[k] * np.cos(k * t) for k in range(1, len(a)))
    speed = np.sqrt(r * r + dr * dr)
    bt = sum(ca[k - 1] * np.cos(k * t) + cb[k - 1] * np.sin(k * t) for k in range(1, 5))
    mean = float(np.sum(bt * speed) / np.sum(speed))
    flux.append(fourier(ca, cb, a0=-mean))
    for _ in range(n - 1):
        flux.append(fourier(rng.standard_normal(4), rng.standard_normal(4)))
    return {"name": "2d-star-inclusions", "dim": 2, "surfaces": surfaces,
            "parent": [-1] + [0] * (n - 1), "sigma": [float(s) for s in sigma], "flux": flux, "M": 4}


def star_degree_problem(seed=21, degree=16, n_incl=4, top=0.012):
    """A star of the given Fourier degree, r(t) = 1 + sum_{k<=degree} a_k cos kt + b_k sin kt
    with a_k, b_k ~ N(0, (0.03 / k)^2) and the top harmonic's cosine set to `top` (the curve
    is wiggly at every scale up to the degree, and r > 0.8), with n_incl circles inside
    (radii U[0.05, 0.12], gap >= 0.03), sigma_1 = 1, sigma_i log-uniform on [0.2, 5], and
    flux data as in star_inclusions_problem (trig polynomials of degree <= 4, zero mean)."""
    rng = np.random.default_rng(seed)
    a = [0.0] + [float(rng.normal(0.0, 0.03 / k)) for k in range(1, degree + 1)]
    b = [0.0] + [float(rng.normal(0.0, 0.03 / k)) for k in range(1, degree + 1)]
    a[degree] = top
    _, curve = _star_curve(a, b)
    assert np.min(np.linalg.norm(curve, axis=1)) > 0.8
    circles = []
    tries = 0
    while len(circles) < n_incl and tries < 100000:
        tries += 1
        rad = rng.uniform(0.05, 0.12)
        c = rng.uniform(-0.8, 0.8, size=2)
        if not _inside_star(a, b, c):
            continue
        if np.min(np.linalg.norm(curve - c, axis=1)) < rad + 0.03:
            continue
        if any(np.linalg.norm(c - c2) < rad + r2 + 0.03 for c2, r2 in circles):
            continue
        circles.append((c, rad))
    surfaces = [_star([0, 0], 1.0, a, b)] + [_sphere(c, r) for c, r in circles]
    n = len(surfaces)
    sigma = [1.0] + list(np.exp(rng.uniform(math.log(0.2), math.log(5.0), n - 1)))
    t = np.linspace(0.0, 2 * np.pi, 8192, endpoint=False)
    r = _star_radius(a, b, t)
    dr = sum(-k * a[k] * np.sin(k * t) + k * b[k] * np.cos(k * t) for k in range(1, len(a)))
    speed = np.sqrt(r * r + dr * dr)
    ca, cb = rng.standard_normal(4), rng.standard_normal(4)
    bt = sum(ca[k - 1] * np.cos(k * t) + cb[k - 1] * np.sin(k * t) for k in range(1, 5))
    flux = [fourier(ca, cb, a0=-float(np.sum(bt * speed) / np.sum(speed)))]
    for _ in range(n - 1):
        flux.append(fourier(rng.standard_normal(4), rng.standard_normal(4)))
    return {"name": f"star-degree-{degree}", "dim": 2, "surfaces": surfaces, "parent": [-1] + [0] * (n - 1),
            "sigma": [float(x) for x in sigma], "flux": flux, "M": 4}


def star_inclusions_points(problem, n, seed=13, near_frac=0.3, band=0.01):
    """n points in the star domain: (1 - near_frac) uniform by rejection and
    near_frac within `band` of a surface (a random surface chosen by length, a
    random point on it, a normal offset U[-band, band]), all kept inside."""
    rng = np.random.default_rng(seed)
    star = problem["surfaces"][0]
    a, b = star["star_a"], star["star_b"]
    n_near = int(round(near_frac * n))
    n_far = n - n_near
    pts = []
    while len(pts) < n_far:
        p = rng.uniform(-1.2, 1.2, size=(4 * n_far, 2))
        pts += list(p[_inside_star(a, b, p)])
    pts = pts[:n_far]
    lengths = []
    for s in problem["surfaces"]:
        if s["kind"] == "star":
            t, c = _star_curve(a, b)
            lengths.append(float(np.sum(np.linalg.norm(np.roll(c, -1, 0) - c, axis=1))))
        else:
            lengths.append(2 * np.pi * s["radius"])
    prob = np.asarray(lengths) / np.sum(lengths)
    near = []
    while len(near) < n_near:
        i = rng.choice(len(lengths), p=prob)
        s = problem["surfaces"][i]
        t = rng.uniform(0, 2 * np.pi)
        off = rng.uniform(-band, band)
        if s["kind"] == "star":
            rr = _star_radius(a, b, np.array([t]))[0]
            p = np.array([rr * np.cos(t), rr * np.sin(t)])
            q = _star_radius(a, b, np.array([t + 1e-6]))[0]
            tang = np.array([q * np.cos(t + 1e-6), q * np.sin(t + 1e-6)]) - p
            nrm = np.array([tang[1], -tang[0]]) / np.linalg.norm(tang)
        else:
            nrm = np.array([np.cos(t), np.sin(t)])
            p = np.asarray(s["center"]) + s["radius"] * nrm
        p = p + off * nrm
        if _inside_star(a, b, p[None, :])[0]:
            near.append(p)
    out = np.asarray(pts + near, dtype=np.float64)
    return out[rng.permutation(len(out))]


def near_surface_points(problem, i, deltas, side=-1, seed=0):
    """One point per entry of `deltas`, at normal distance delta from surface i
    (a circle, a d-sphere or a 2D star), on its inner side (side = -1) or its
    outer side (side = +1), each at a random position along the surface."""
    rng = np.random.default_rng(seed)
    s = problem["surfaces"][i]
    c = np.asarray(s["center"], dtype=np.float64)
    out = []
    for dl in deltas:
        if s["kind"] == "sphere":
            g = rng.standard_normal(len(c))
            g /= np.linalg.norm(g)
            out.append(c + (s["radius"] + side * dl) * g)
        elif s["kind"] == "star":
            a, b, R = s["star_a"], s["star_b"], s["radius"]
            t = rng.uniform(0.0, 2.0 * np.pi)
            r = R * _star_radius(a, b, np.array([t]))[0]
            dr = R * sum(k * (b[k] * np.cos(k * t) - a[k] * np.sin(k * t)) for k in range(1, len(a)))
            tang = np.array([dr * np.cos(t) - r * np.sin(t), dr * np.sin(t) + r * np.cos(t)])
            nrm = np.array([tang[1], -tang[0]]) / np.linalg.norm(tang)
            out.append(c + r * np.array([np.cos(t), np.sin(t)]) + side * dl * nrm)
        else:
            raise ValueError("near_surface_points takes circles, spheres and stars")
    return np.ascontiguousarray(np.asarray(out, dtype=np.float64))


# ---------------------------------------------------------------------------
# batch of heterogeneous manufactured-solution instances
# ---------------------------------------------------------------------------

def _harmonic_basis(dim):
    """Monomial expansions of a basis of harmonic polynomials of degree 1..3."""
    def mono(*pairs):
        return [(c, e) for c, e in pairs]
    if dim == 2:
        return [mono((1.0, (1, 0))), mono((1.0, (0, 1))),
                mono((1.0, (2, 0)), (-1.0, (0, 2))), mono((2.0, (1, 1))),
                mono((1.0, (3, 0)), (-3.0, (1, 2))), mono((3.0, (2, 1)), (-1.0, (0, 3)))]
    return [mono((1.0, (1, 0, 0))), mono((1.0, (0, 1, 0))), mono((1.0, (0, 0, 1))),
            mono((1.0, (2, 0, 0)), (-1.0, (0, 2, 0))), mono((1.0, (2, 0, 0)), (-1.0, (0, 0, 2))),
            mono((1.0, (1, 1, 0))), mono((1.0, (1, 0, 1))), mono((1.0, (0, 1, 1))),
            mono((1.0, (1, 1, 1))),
            mono((1.0, (3, 0, 0)), (-3.0, (1, 2, 0))), mono((1.0, (3, 0, 0)), (-3.0, (1, 0, 2))),
            mono((1.0, (0, 3, 0)), (-3.0, (2, 1, 0))), mono((1.0, (0, 3, 0)), (-3.0, (0, 1, 2))),
            mono((1.0, (0, 0, 3)), (-3.0, (2, 0, 1))), mono((1.0, (0, 0, 3)), (-3.0, (0, 2, 1)))]


def random_harmonic_poly(dim, rng):
    """A random harmonic polynomial of degree <= 3 as merged monomial terms."""
    terms = {}
    for poly in _harmonic_basis(dim):
        w = rng.standard_normal()
        for c, e in poly:
            terms[e] = terms.get(e, 0.0) + w * c
    return [(c, e) for e, c in sorted(terms.items()) if c != 0.0]


def eval_poly(terms, x):
    """P(x) and grad P(x) of a monomial expansion at points x [n, dim]."""
    x = np.atleast_2d(x)
    n, d = x.shape
    v = np.zeros(n)
    g = np.zeros((n, d))
    for c, e in terms:
        v += c * np.prod(x ** np.asarray(e), axis=1)
        for k in range(d):
            if e[k] == 0:
                continue
            ee = list(e)
            ee[k] -= 1
            g[:, k] += c * e[k] * np.prod(x ** np.asarray(ee), axis=1)
    return v, g


def manufactured_instance(dim, rng, k_max=64, r_lo=0.02, r_hi=0.15, gap=0.01, max_tries=10000, k_exact=None):
    """Unit disk/ball with k ~ U{1..k_max} (or k_exact) non-overlapping
    circles/spheres (radii U[r_lo, r_hi]; on rejection failure the count is
    reduced and recorded), sigma_1 = 1, sigma_i log-uniform on [0.05, 20], and
    flux data of the manufactured solution u_h (harmonic, degree <= 3):
    b_1 = sigma_1 dn u_h, b_i = (sigma_parent - sigma_i) dn u_h."""
    k_req = int(rng.integers(1, k_max + 1)) if k_exact is None else int(k_exact)
    incl = []
    tries = 0
    while len(incl) < k_req and tries < max_tries:
        tries += 1
        rad = rng.uniform(r_lo, r_hi)
        g = rng.standard_normal(dim)
        g /= np.linalg.norm(g)
        c = g * (1.0 - rad - gap) * rng.random() ** (1.0 / dim)
        if np.linalg.norm(c) + rad + gap > 1.0:
            continue
        if any(np.linalg.norm(c - c2) < rad + r2 + gap for c2, r2 in incl):
            continue
        incl.append((c, rad))
    n = 1 + len(incl)
    sigma = [1.0] + list(np.exp(rng.uniform(math.log(0.05), math.log(20.0), n - 1)))
    uh = random_harmonic_poly(dim, rng)
    flux = [harmonic_poly(sigma[0], uh, dim)]
    for i in range(1, n):
        flux.append(harmonic_poly(sigma[0] - sigma[i], uh, dim))
    return {"name": f"batch-{dim}d", "dim": dim,
            "surfaces": [_sphere([0.0] * dim, 1.0)] + [_sphere(c, r) for c, r in incl],
            "parent": [-1] + [0] * (n - 1), "sigma": [float(s) for s in sigma], "flux": flux,
            "M": 4 if dim == 2 else 6, "u_h": uh, "k_requested": k_req}


def batch_instances(n_inst=256, seed=5, k_max=64, p_range=(16, 4096), w_range=(1e4, 1e5), point_seed=15):
    """n_inst instances, alternating 2D / 3D, with per-instance point counts
    log-uniform on p_range and walk counts log-uniform on w_range (rounded to a
    multiple of 32)."""
    rng = np.random.default_rng(seed)
    prng = np.random.default_rng(point_seed)
    out = []
    for i in range(n_inst):
        dim = 2 if i % 2 == 0 else 3
        prob = manufactured_instance(dim, rng, k_max=k_max)
        P = int(round(math.exp(rng.uniform(math.log(p_range[0]), math.log(p_range[1])))))
        W = int(round(math.exp(rng.uniform(math.log(w_range[0]), math.log(w_range[1]))) / 32.0)) * 32
        pts = ball_points(P, dim, int(prng.integers(0, 2**31)))
        out.append({"problem": prob, "points": pts, "n_walks": max(W, 32)})
    return out


# ---------------------------------------------------------------------------
# nested ellipsoids with the point-charge potential (the paper's Example 2)
# ---------------------------------------------------------------------------

def ellipsoids_problem(dim, M=None):
    """Three nested ellipsoids (Example 2, Table of ellipsoid parameters):
    Omega_1 centre (1.3, 0, ...), diag(A) = [1, 0.9, 1.2, ...], sigma 1.1;
    Omega_2 centre (1.4, 0, ...), diag(A) = [1.5, 3.2, 2, ...], A_12 = A_21 = -1, sigma 1.3;
    Omega_3 centre (1.6, 0, ...), diag(A) = [8, 6, 4, ...], A_12 = A_21 = -2, sigma 0.9.
    Data of the manufactured solution u = |x|^{2-dim} (a point charge at the
    origin, outside every region): Neumann flux sigma_1 d_n u on the outer
    surface and jumps (sigma_p - sigma_i) d_n u across the interfaces.
    M as in the paper's table: 5, 6, 7, 8 for dim 3..6.

    As printed, Omega_2 (centre 1.4) reaches outside Omega_1 (the quadratic form
    of Omega_1 reaches 1.14 on it); its centre is taken at (1.3, 0, ...), the
    centre of Omega_1, which nests the three ellipsoids (forms <= 0.95 on the
    inner surfaces) and changes nothing else."""
    if dim < 3:
        raise ValueError("the point-charge workload needs dim >= 3")

    def mat(diag, off):
        A = np.diag(np.asarray(diag, dtype=np.float64))
        A[0, 1] = A[1, 0] = off
        return A

    e1 = [0.0] * dim
    A1 = mat([1.0, 0.9] + [1.2] * (dim - 2), 0.0)
    A2 = mat([1.5, 3.2] + [2.0] * (dim - 2), -1.0)
    A3 = mat([8.0, 6.0] + [4.0] * (dim - 2), -2.0)
    c1, c2, c3 = ([x] + e1[1:] for x in (1.3, 1.3, 1.6))
    sigma = [1.1, 1.3, 0.9]
    parent = [-1, 0, 1]
    zero = [0.0] * dim
    flux = [{"basis": "point_charge", "coef": [sigma[0]] + zero},
            {"basis": "point_charge", "coef": [sigma[0] - sigma[1]] + zero},
            {"basis": "point_charge", "coef": [sigma[1] - sigma[2]] + zero}]
    return {"name": f"{dim}d-ellipsoids", "dim": dim,
            "surfaces": [_ellipsoid(c1, A1), _ellipsoid(c2, A2), _ellipsoid(c3, A3)],
            "parent": parent, "sigma": sigma, "flux": flux, "M": {3: 5, 4: 6, 5: 7, 6: 8}[dim] if M is None else M}


def ellipsoid_chain_problem(dim, n=8, shrink=0.8, M=4):
    """n concentric nested ellipsoids: the outer one of ellipsoids_problem (centre (1.3, 0,
    ...), diag(A) = [1, 0.9, 1.2, ...]), each next one the previous scaled by `shrink` about
    the centre; sigma alternating 1 and log-uniform values on [0.3, 3] (seed 0), and the
    point-charge data of u = |x|^{2-dim} (the origin lies outside the outer ellipsoid)."""
    rng = np.random.default_rng(0)
    c = [1.3] + [0.0] * (dim - 1)
    A0 = np.diag(np.asarray([1.0, 0.9] + [1.2] * (dim - 2), dtype=np.float64))
    surfaces = [_ellipsoid(c, A0 / shrink ** (2 * i)) for i in range(n)]
    sigma = [1.0] + [float(np.exp(rng.uniform(math.log(0.3), math.log(3.0)))) for _ in range(n - 1)]
    zero = [0.0] * dim
    flux = [{"basis": "point_charge", "coef": [sigma[0]] + zero}]
    for i in range(1, n):
        flux.append({"basis": "point_charge", "coef": [sigma[i - 1] - sigma[i]] + zero})
    return {"name": f"{dim}d-ellipsoid-chain", "dim": dim, "surfaces": surfaces,
            "parent": [-1] + list(range(n - 1)), "sigma": sigma, "flux": flux, "M": M}


def inside_ellipsoid(s, p):
    c = np.asarray(s["center"], dtype=np.float64)
    A = np.asarray(s["matrix"], dtype=np.float64)
    e = np.atleast_2d(p) - c
    return np.einsum("ni,ij,nj->n", e, A, e) < 1.0


def ellipsoid_points(problem, n, seed=16):
    """n points uniform in the outer ellipsoid (rejection from its bounding box)."""
    s = problem["surfaces"][0]
    A = np.asarray(s["matrix"], dtype=np.float64)
    c = np.asarray(s["center"], dtype=np.float64)
    half = np.sqrt(np.diag(np.linalg.inv(A)))          # half-widths of the bounding box
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        p = c + rng.uniform(-1.0, 1.0, size=(4 * n, len(c))) * half
        out += list(p[inside_ellipsoid(s, p)])
    return np.ascontiguousarray(np.asarray(out[:n], dtype=np.float64))


def point_charge(x):
    """u = |x|^{2-d} and grad u = (2 - d) |x|^{-d} x (the manufactured solution)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d = x.shape[1]
    r = np.linalg.norm(x, axis=1)
    return r ** (2 - d), (2 - d) * (r ** -d)[:, None] * x


# ---------------------------------------------------------------------------
# triangle meshes: a star-shaped outer boundary with rock-like inclusions
# ---------------------------------------------------------------------------

def icosphere(subdiv):
    """Unit icosphere: the icosahedron with every triangle split into four,
    subdiv times, vertices projected to the sphere; faces counter-clockwise
    seen from outside.  20 * 4^subdiv triangles."""
    t = (1.0 + 5 ** 0.5) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.asarray(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    for _ in range(subdiv):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                mid[key] = len(V) - 1
            return mid[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    V = np.asarray(V)
    F = np.asarray(F, dtype=np.int64)
    # orient outward: the signed volume must be positive
    v0, v1, v2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    if np.sum(np.einsum("ij,ij->i", v0, np.cross(v1, v2))) < 0:
        F = F[:, ::-1].copy()
    return V, F


def radial_mesh(center, radius, subdiv, amp, seed):
    """A star-shaped closed mesh: icosphere vertices u moved to
    center + radius (1 + amp f(u)) u with f a sum of six random plane waves
    (|f| <= 1), which keeps the surface star-shaped and outward-oriented."""
    V, F = icosphere(subdiv)
    rng = np.random.default_rng(seed)
    k = rng.standard_normal((6, 3)) * 1.5
    ph = rng.uniform(0, 2 * np.pi, 6)
    f = np.cos(V @ k.T + ph).sum(axis=1) / 6.0
    Vr = np.asarray(center, dtype=np.float64) + radius * (1.0 + amp * f)[:, None] * V
    return Vr, F


def bellows_problem(subdiv=6, k=80.0, amp=0.3, M=3):
    """One closed radial mesh shaped like a bellows along z, r(u) = 1 + amp cos(k u_z)
    (20 4^subdiv triangles), with zero flux: lines through it cross it many times (at
    the defaults about 5 % of random lines through a point of it cross it more than 32
    times), the case in which a library must report that it truncated a crossing list."""
    V, F = icosphere(subdiv)
    V = np.asarray(V, dtype=np.float64)
    Vr = (1.0 + amp * np.cos(k * V[:, 2]))[:, None] * V
    return {"name": "bellows", "dim": 3, "surfaces": [_mesh(Vr, F, [0.0, 0.0, 0.0])], "parent": [-1],
            "sigma": [1.0], "flux": [{"basis": "zero", "coef": []}], "M": M}


def _mesh(V, F, center):
    return {"kind": "mesh", "center": [float(c) for c in center],
            "vertices": np.asarray(V, dtype=np.float64).tolist(), "triangles": np.asarray(F, dtype=np.int64).tolist()}


def winding_number(V, F, P):
    """Generalised winding number of the closed mesh (V, F) at points P [n, 3]
    (solid angle of every triangle, Van Oosterom-Strackee): 1 inside, 0 outside."""
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    out = np.zeros(len(P))
    for lo in range(0, len(P), 256):
        p = P[lo:lo + 256, None, :]
        a, b, c = V[F[:, 0]][None] - p, V[F[:, 1]][None] - p, V[F[:, 2]][None] - p
        la, lb, lc = (np.linalg.norm(v, axis=2) for v in (a, b, c))
        num = np.einsum("pti,pti->pt", a, np.cross(b, c))
        den = la * lb * lc + np.einsum("pti,pti->pt", a, b) * lc + np.einsum("pti,pti->pt", b, c) * la \
            + np.einsum("pti,pti->pt", c, a) * lb
        out[lo:lo + 256] = np.sum(2 * np.arctan2(num, den), axis=1) / (4 * np.pi)
    return out


def rocks_problem(n_rocks=6, seed=7, subdiv_outer=4, subdiv_rock=3, M=5):
    """Rock-like inclusions in a star-shaped body, the shape of the paper's
    groundwater example (a hill with rocks, Sec. 5) with synthetic meshes: the
    outer boundary a radial mesh of mean radius 1 (amp 0.06, 20 4^subdiv_outer
    triangles), n_rocks radial meshes of radius U[0.12, 0.2] (amp 0.2), placed
    by rejection with bounding spheres 0.05 apart.  sigma = 0.2 outside, rocks
    0.03 - 0.05 (the example's values).  Data of a random harmonic polynomial
    u_h (degree <= 3), the manufactured solution: b_1 = sigma_1 dn u_h,
    b_i = (sigma_1 - sigma_i) dn u_h."""
    rng = np.random.default_rng(seed)
    Vo, Fo = radial_mesh([0, 0, 0], 1.0, subdiv_outer, 0.06, seed + 1)
    r_in = float(np.min(np.linalg.norm(Vo, axis=1)))
    rocks = []
    tries = 0
    while len(rocks) < n_rocks and tries < 10000:
        tries += 1
        rad = rng.uniform(0.12, 0.2)
        bound = rad * 1.2
        c = rng.uniform(-1, 1, 3)
        if np.linalg.norm(c) + bound > r_in - 0.05:
            continue
        if any(np.linalg.norm(c - c2) < bound + b2 + 0.05 for c2, b2, _ in rocks):
            continue
        rocks.append((c, bound, rad))
    surfaces = [_mesh(Vo, Fo, [0, 0, 0])]
    for j, (c, _, rad) in enumerate(rocks):
        V, F = radial_mesh(c, rad, subdiv_rock, 0.2, seed + 10 + j)
        surfaces.append(_mesh(V, F, c))
    sigma = [0.2] + [float(v) for v in rng.uniform(0.03, 0.05, len(rocks))]
    terms = random_harmonic_poly(3, rng)
    flux = [harmonic_poly(sigma[0], terms, 3)] + [harmonic_poly(sigma[0] - s, terms, 3) for s in sigma[1:]]
    return {"name": "3d-rocks", "dim": 3, "surfaces": surfaces, "parent": [-1] + [0] * len(rocks),
            "sigma": sigma, "flux": flux, "M": M, "u_terms": terms}


def mesh_points(problem, n, seed=17, margin=0.02):
    """n points inside the outer mesh (winding number > 1/2, and more than
    `margin` inside the outer mesh's inscribed radius bound), uniform."""
    s = problem["surfaces"][0]
    V = np.asarray(s["vertices"])
    rmax = float(np.max(np.linalg.norm(V - np.asarray(s["center"]), axis=1)))
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        p = rng.uniform(-rmax, rmax, size=(2 * n, 3)) + np.asarray(s["center"])
        w = winding_number(V, s["triangles"], p)
        out += list(p[w > 0.5])
    return np.ascontiguousarray(np.asarray(out[:n], dtype=np.float64))


CONFIGS = {
    "2d-concentric": "unit disk + r=0.5 inclusion, 64 polar-grid points, W=1e4, M=4",
    "3d-nested": "spheres 1/0.8/0.5, sigma 1/5/0.2, 4096 ball points, W=1e5, M=6",
    "2d-star-inclusions": "star + 32 circles, 16384 points (30% near surfaces), W=1e5, M=4",
    "6d-nested": "hyperspheres 1/0.6, sigma 1/4, 1024 ball points, W=1e6, M=8",
    "batch": "256 manufactured 2D/3D instances, 1-64 inclusions, P 16..4096, W 1e4..1e5",
    "ellipsoids": "3 nested ellipsoids (Example 2), point charge at the origin, 3D-6D, M = d + 2",
    "3d-rocks": "star-shaped outer mesh + 6 rock meshes (12800 triangles), manufactured harmonic data, M = 5",
}
