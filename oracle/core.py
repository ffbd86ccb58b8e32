"""Plain FP64 CPU oracle of the Walk-on-Interfaces estimator (arXiv 2508.16767).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this module; the product path never does.  It
shares no code with the CUDA library.

The walk itself (Algorithms 1-3) runs in the plain C file woi_oracle.c; this
module prepares its inputs from a problem dictionary with numpy/scipy:

  * Sec. 3: alpha_1 = 2, alpha_i = 2 (sigma_i - sigma_{p_i}) / (sigma_{p_i} + sigma_i),
    beta_1 = (2 / sigma_1) b_1, beta_i = -2 b_i / (sigma_{p_i} + sigma_i);
  * Thm 4.2, Eq. scheduled_interface_pdf: P(H_i = n) = |alpha_n| / ||alpha||_1,
    turned into integer thresholds T_n = floor(2^32 C_n / A), C_n the cumulative
    sum of |alpha| in surface order and A = ||alpha||_1 (T_N = 2^32);
  * Sec. 1: the tree (strict-descendant relation) from the parent array;
  * |dOmega_i| (circle / d-sphere closed form, star by Gauss-Legendre quadrature,
    ellipsoid by a one-dimensional integral for the mean area ratio, see
    ellipsoid_area);
  * ellipsoids (Sec. 5, Example 2): the symmetric square root A^{-1/2} that
    maps the unit sphere onto the surface, and sqrt of the largest eigenvalue;
  * triangle meshes (3D): per triangle v0, e1, e2 and the unit normal of e1 x e2,
    the area as the sum of the triangle areas, and the cumulative-area
    thresholds floor(2^32 C_j / A) that pick a triangle by area;
  * Sec. 4.4: the beta >= 0 / beta < 0 arcs of 2D surfaces for the variance-
    reduced estimator, by a dense sign scan and Brent's method; in d >= 3 the
    hemispheres of data linear in the unit vector.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys

import numpy as np
from scipy import integrate, optimize

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "woi_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")

MAX_DIM = 6
MAX_STAR = 16
STAR_PANELS = 256
STAR_SCAN = 4096
SPHERE, STAR, ELLIPSOID, MESH = 0, 1, 2, 3
KIND = {"sphere": SPHERE, "star": STAR, "ellipsoid": ELLIPSOID, "mesh": MESH}
FLUX = {"zero": 0, "fourier": 1, "real_sh": 2, "harmonic_poly": 3, "point_charge": 4}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over points)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB)
        P = ctypes.POINTER
        _lib.or_estimate.argtypes = [P(OrProblem), P(OrOpts), ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_estimate.restype = ctypes.c_int
        _lib.or_walks.argtypes = [P(OrProblem), P(OrOpts), ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_set_mutant.argtypes = [ctypes.c_int]
        _lib.or_set_mutant_bound.argtypes = [ctypes.c_int]
        _lib.or_set_perturb.argtypes = [ctypes.c_double]
        _lib.or_threads.argtypes = [ctypes.c_int]
        _lib.or_threads.restype = ctypes.c_int
        _lib.or_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_test_real_sh.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        _lib.or_test_real_sh.restype = ctypes.c_double
        _lib.or_test_star_arclen.argtypes = [P(OrProblem), ctypes.c_int, ctypes.c_double]
        _lib.or_test_star_arclen.restype = ctypes.c_double
        _lib.or_test_intersections.argtypes = [P(OrProblem), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        _lib.or_test_intersections.restype = ctypes.c_int
        _lib.or_test_flux.argtypes = [P(OrProblem), ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        _lib.or_test_flux.restype = ctypes.c_double
        _lib.or_test_uniform_point.argtypes = [P(OrProblem), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        _lib.or_test_uniform_part_point.argtypes = [P(OrProblem), ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                    ctypes.c_uint64, ctypes.c_void_p]
        _lib.or_test_direction.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                           ctypes.c_void_p]
    return _lib


class OrProblem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_surf", ctypes.c_int)] + [
        (n, ctypes.c_void_p) for n in
        ["type", "center", "radius", "star_K", "star_a", "star_b", "star_s", "star_scan", "area", "is_desc",
         "alpha",
         "beta_scale", "thresh"]] + [("alpha_l1", ctypes.c_double)] + [
        (n, ctypes.c_void_p) for n in
        ["flux_basis", "flux_off", "flux_n", "flux_coef", "arc_off", "arc_n", "arc_t0", "arc_t1", "arc_sign",
         "arc_len", "part_len", "ell_A", "ell_map", "ell_jmax", "mesh_off", "mesh_n", "tri", "tri_thresh"]]


class OrOpts(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("variant", ctypes.c_int), ("sched_group", ctypes.c_int)]


def set_mutant(m: int) -> None:
    """Plant one of the numbered mistakes in the C oracle (tests only; 0 = none)."""
    lib().or_set_mutant(int(m))


def set_mutant_bound(m: int) -> None:
    """Plant a mistake in the per-walk error bound (tests only; 1 drops the states'
    term, 0 = none)."""
    lib().or_set_mutant_bound(int(m))


def set_perturb(rel: float) -> None:
    """Move every walk state y on surface s by rel |y - c_s| and the evaluation
    point by rel |x - c_s| per tally (tests of the error bound only; 0 = exact)."""
    lib().or_set_perturb(float(rel))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


# ---------------------------------------------------------------------------
# Sec. 3 coefficients and the schedule
# ---------------------------------------------------------------------------

def alpha_beta_scale(sigma, parent):
    """alpha_i and the factor beta_i / b_i of the unit-coefficient system (Sec. 3)."""
    n = len(sigma)
    alpha = np.zeros(n)
    bscale = np.zeros(n)
    for i in range(n):
        if parent[i] < 0:
            alpha[i] = 2.0
            bscale[i] = 2.0 / sigma[i]
        else:
            sp, si = sigma[parent[i]], sigma[i]
            alpha[i] = 2.0 * (si - sp) / (sp + si)
            bscale[i] = -2.0 / (sp + si)
    return alpha, bscale


def schedule_thresholds(alpha):
    """Integer thresholds of P(H_i = n) = |alpha_n| / ||alpha||_1 (Thm 4.2):
    H = min{n : w < T_n} for a 32-bit word w; T_n = floor(2^32 C_n / A)."""
    absa = np.abs(np.asarray(alpha, dtype=np.float64))
    A = 0.0
    for v in absa:
        A += v
    out = np.zeros(len(absa), dtype=np.uint64)
    C = 0.0
    for n, v in enumerate(absa):
        C += v
        out[n] = np.uint64(math.floor(math.ldexp(C / A, 32)))
    out[-1] = np.uint64(1 << 32)
    return out, A


def descendant_matrix(parent):
    n = len(parent)
    m = np.zeros((n, n), dtype=np.int32)
    for a in range(n):
        p = parent[a]
        while p >= 0:
            m[a, p] = 1
            p = parent[p]
    return m


def omega(d):
    """|S^{d-1}| = d alpha(d) (Sec. 2)."""
    return 2.0 * math.pi ** (d / 2) / math.gamma(d / 2)


# ---------------------------------------------------------------------------
# star curves
# ---------------------------------------------------------------------------

def star_r(s, t):
    R = s["radius"]
    a, b = s["star_a"], s["star_b"]
    v = 1.0
    dv = 0.0
    for k in range(1, len(a)):
        v += a[k] * math.cos(k * t) + b[k] * math.sin(k * t)
        dv += k * (-a[k] * math.sin(k * t) + b[k] * math.cos(k * t))
    return R * v, R * dv


def star_speed(s, t):
    r, dr = star_r(s, t)
    return math.hypot(r, dr)


_GL_X, _GL_W = np.polynomial.legendre.leggauss(40)


def star_length(s, a, b):
    """int_a^b |gamma'(t)| dt by 40-point Gauss-Legendre on panels of width <= 2 pi / 256
    (machine precision for the smooth integrands of star curves)."""
    n = max(1, int(math.ceil((b - a) / (2 * math.pi / STAR_PANELS))))
    tot = 0.0
    for j in range(n):
        lo = a + (b - a) * j / n
        hi = a + (b - a) * (j + 1) / n
        t = 0.5 * (hi - lo) * _GL_X + 0.5 * (hi + lo)
        tot += 0.5 * (hi - lo) * float(np.sum(_GL_W * np.array([star_speed(s, x) for x in t])))
    return tot


def star_arclen_panels(s):
    """Arc length at t_j = 2 pi j / STAR_PANELS."""
    out = np.zeros(STAR_PANELS + 1)
    h = 2 * math.pi / STAR_PANELS
    for j in range(STAR_PANELS):
        out[j + 1] = out[j] + star_length(s, j * h, (j + 1) * h)
    return out


def ellipsoid_axes(s):
    """Eigen-decomposition of the ellipsoid matrix: A = R diag(lam) R^T, semi-axes
    a = lam^{-1/2}; y = c + R diag(a) u maps the unit sphere onto the surface."""
    A = np.asarray(s["matrix"], dtype=np.float64)
    lam, R = np.linalg.eigh(0.5 * (A + A.T))
    if np.any(lam <= 0):
        raise ValueError("ellipsoid matrix must be positive definite")
    return lam, R


def ellipsoid_area(dim, lam):
    """|dE| for E = {y : y^T A y <= 1} with eigenvalues lam of A.

    The map u -> diag(a) u (a = lam^{-1/2}) takes the unit sphere onto dE and
    scales area by J(u) prod(a), J(u) = |diag(sqrt(lam)) u|, so |dE| =
    |S^{d-1}| prod(a) E_u[J].  With a standard normal g = |g| u (|g| and u
    independent), E_u[J] = E sqrt(S) / E|g| for S = sum lam_k g_k^2, and
    sqrt(S) = (1 / (2 sqrt(pi))) int_0^inf (1 - exp(-s S)) s^{-3/2} ds gives
    E sqrt(S) = (1 / sqrt(pi)) int_0^inf (1 - prod_k (1 + 2 lam_k t^2)^{-1/2}) t^{-2} dt
    (s = t^2, E exp(-s lam g^2) = (1 + 2 s lam)^{-1/2}); E|g| = sqrt(2) Gamma((d+1)/2) / Gamma(d/2)."""
    lam = np.asarray(lam, dtype=np.float64)

    def f(t):
        if t == 0.0:
            return float(np.sum(lam))
        # 1 - prod (1 + x_k)^{-1/2} without cancellation at small t
        return -math.expm1(-0.5 * float(np.sum(np.log1p(2.0 * lam * t * t)))) / (t * t)

    scale = 1.0 / math.sqrt(float(np.max(lam)))
    I1, _ = integrate.quad(f, 0.0, 50.0 * scale, epsabs=0, epsrel=1e-13, limit=500)
    I2, _ = integrate.quad(f, 50.0 * scale, np.inf, epsabs=0, epsrel=1e-13, limit=500)
    e_sqrt_s = (I1 + I2) / math.sqrt(math.pi)
    e_norm = math.sqrt(2.0) * math.exp(math.lgamma((dim + 1) / 2) - math.lgamma(dim / 2))
    return omega(dim) * float(np.prod(lam ** -0.5)) * e_sqrt_s / e_norm


def mesh_triangles(s):
    """[n, 12] rows (v0, e1, e2, unit normal of e1 x e2) and the triangle areas,
    with the cross product and its length written out (no library norm)."""
    V = np.asarray(s["vertices"], dtype=np.float64)
    F = np.asarray(s["triangles"], dtype=np.int64)
    v0, v1, v2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    e1, e2 = v1 - v0, v2 - v0
    cx = e1[:, 1] * e2[:, 2] - e1[:, 2] * e2[:, 1]
    cy = e1[:, 2] * e2[:, 0] - e1[:, 0] * e2[:, 2]
    cz = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    ln = np.sqrt(cx * cx + cy * cy + cz * cz)
    n = np.stack([cx / ln, cy / ln, cz / ln], axis=1)
    return np.concatenate([v0, e1, e2, n], axis=1), 0.5 * ln


def mesh_thresholds(areas):
    """P(triangle j) = area_j / A as 32-bit thresholds T_j = floor(2^32 C_j / A), T_last = 2^32."""
    A = 0.0
    for a in areas:
        A += float(a)
    out = np.zeros(len(areas), dtype=np.uint64)
    C = 0.0
    for j, a in enumerate(areas):
        C += float(a)
        out[j] = np.uint64(math.floor(math.ldexp(C / A, 32)))
    out[-1] = np.uint64(1 << 32)
    return out, A


def surface_area(dim, s):
    if s["kind"] == "mesh":
        return mesh_thresholds(mesh_triangles(s)[1])[1]
    if s["kind"] == "sphere":
        return omega(dim) * s["radius"] ** (dim - 1)
    if s["kind"] == "ellipsoid":
        return ellipsoid_area(dim, ellipsoid_axes(s)[0])
    return float(star_arclen_panels(s)[-1])


# ---------------------------------------------------------------------------
# flux (host-side evaluation used by the variance-reduction arcs)
# ---------------------------------------------------------------------------

def fourier_eval(coef, t):
    v = coef[0] * np.ones_like(t)
    K = (len(coef) - 1) // 2
    for k in range(1, K + 1):
        v = v + coef[2 * k - 1] * np.cos(k * t) + coef[2 * k] * np.sin(k * t)
    return v


def linear_on_sphere(dim, s, flux):
    """Data whose value on the sphere is linear in the unit vector u (degree-1 real
    harmonics, harmonic polynomials of degree 1): its sign parts are hemispheres."""
    if s["kind"] != "sphere":
        return False
    if flux["basis"] == "real_sh":
        return dim == 3 and all(v == 0.0 for i, v in enumerate(flux["coef"]) if not 1 <= i <= 3)
    if flux["basis"] == "harmonic_poly":
        c = flux["coef"]
        T = int(c[1])
        return all(sum(c[2 + t * (dim + 1) + 1: 2 + (t + 1) * (dim + 1)]) <= 1 for t in range(T))
    return False


def vr_parts(dim, s, flux):
    """|dOmega^+|, |dOmega^-| in d >= 3 (Sec. 4.4): zero data puts the whole surface in the
    beta >= 0 part; data linear in u splits a sphere into two hemispheres; other data, and
    every ellipsoid and mesh, has parts of no closed form, marked (-1, -1): the start is
    then drawn from uniform trials weighted by their fraction of each sign."""
    A = surface_area(dim, s)
    if flux["basis"] == "zero":
        return (A, 0.0)
    if linear_on_sphere(dim, s, flux):
        return (0.5 * A, 0.5 * A)
    return (-1.0, -1.0)


def vr_arcs(dim, s, flux, bscale, n_scan=20000):
    """Arcs of dOmega^+ = {beta >= 0} and dOmega^- = {beta < 0} (Sec. 4.4) of a
    2D surface with Fourier flux, cut at t = 0 and at every sign change."""
    if dim != 2:
        return None
    basis = flux["basis"]
    if basis == "zero":
        L = surface_area(dim, s)
        return [(0.0, 2 * math.pi, 1, L)]
    if basis != "fourier":
        return None
    coef = np.asarray(flux["coef"], dtype=np.float64)

    def beta(t):
        return bscale * fourier_eval(coef, np.asarray(t, dtype=np.float64))

    t = np.linspace(0.0, 2 * math.pi, n_scan + 1)
    f = beta(t)
    roots = []
    for j in range(n_scan):
        if (f[j] < 0) != (f[j + 1] < 0):
            roots.append(optimize.brentq(lambda x: float(beta(x)), t[j], t[j + 1], xtol=1e-15, rtol=1e-15))
    cuts = [0.0] + roots + [2 * math.pi]
    arcs = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b <= a:
            continue
        sign = 1 if float(beta(0.5 * (a + b))) >= 0 else -1
        if s["kind"] == "sphere":
            L = s["radius"] * (b - a)
        else:
            L = star_length(s, a, b)
        arcs.append((a, b, sign, L))
    return arcs


# ---------------------------------------------------------------------------
# the ctypes problem
# ---------------------------------------------------------------------------

class Prepared:
    """Arrays of a problem in the oracle's layout; keeps them alive."""

    def __init__(self, problem, variant="plain"):
        d = int(problem["dim"])
        surfs = problem["surfaces"]
        n = len(surfs)
        parent = [int(p) for p in problem["parent"]]
        sigma = [float(s) for s in problem["sigma"]]
        self.dim, self.n = d, n
        self.type = np.array([KIND[s["kind"]] for s in surfs], dtype=np.int32)
        self.center = np.zeros((n, MAX_DIM))
        self.radius = np.array([s.get("radius", 0.0) for s in surfs], dtype=np.float64)
        self.ell_A = np.zeros((n, MAX_DIM, MAX_DIM))
        self.ell_map = np.zeros((n, MAX_DIM, MAX_DIM))
        self.ell_jmax = np.zeros(n)
        self.mesh_off = np.zeros(n, dtype=np.int32)
        self.mesh_n = np.zeros(n, dtype=np.int32)
        tris, thr = [np.zeros((0, 12))], [np.zeros(0, dtype=np.uint64)]
        for i, s in enumerate(surfs):
            if s["kind"] == "mesh":
                if d != 3:
                    raise ValueError("meshes are 3D surfaces")
                T, ar = mesh_triangles(s)
                self.mesh_off[i] = sum(len(t) for t in tris)
                self.mesh_n[i] = len(T)
                tris.append(T)
                thr.append(mesh_thresholds(ar)[0])
        self.tri = np.ascontiguousarray(np.concatenate(tris + [np.zeros((1, 12))]))
        self.tri_thresh = np.ascontiguousarray(np.concatenate(thr + [np.zeros(1, dtype=np.uint64)]))
        self.star_K = np.zeros(n, dtype=np.int32)
        self.star_a = np.zeros((n, MAX_STAR + 1))
        self.star_b = np.zeros((n, MAX_STAR + 1))
        self.star_s = np.zeros((n, STAR_PANELS + 1))
        self.star_scan = np.zeros((n, STAR_SCAN + 1, 2))
        for i, s in enumerate(surfs):
            self.center[i, :d] = s["center"]
            if s["kind"] == "ellipsoid":
                lam, R = ellipsoid_axes(s)
                self.ell_A[i, :d, :d] = np.asarray(s["matrix"], dtype=np.float64)
                self.ell_map[i, :d, :d] = (R * (lam ** -0.5)[None, :]) @ R.T     # A^{-1/2}
                self.ell_jmax[i] = math.sqrt(float(np.max(lam)))
            if s["kind"] == "star":
                K = len(s["star_a"]) - 1
                self.star_K[i] = K
                self.star_a[i, :K + 1] = s["star_a"]
                self.star_b[i, :K + 1] = s["star_b"]
                self.star_s[i] = star_arclen_panels(s)
                for j in range(STAR_SCAN + 1):
                    th = 2 * math.pi * j / STAR_SCAN
                    r, _ = star_r(s, th)
                    self.star_scan[i, j] = [s["center"][0] + r * math.cos(th), s["center"][1] + r * math.sin(th)]
        self.area = np.array([self.star_s[i, -1] if surfs[i]["kind"] == "star" else surface_area(d, surfs[i])
                              for i in range(n)])
        self.is_desc = descendant_matrix(parent)
        self.alpha, self.beta_scale = alpha_beta_scale(sigma, parent)
        self.thresh, self.alpha_l1 = schedule_thresholds(self.alpha)
        fl = problem["flux"]
        self.flux_basis = np.array([FLUX[f["basis"]] for f in fl], dtype=np.int32)
        self.flux_n = np.array([len(f["coef"]) for f in fl], dtype=np.int32)
        self.flux_off = np.concatenate([[0], np.cumsum(self.flux_n)[:-1]]).astype(np.int32)
        self.flux_coef = np.concatenate([np.asarray(f["coef"], dtype=np.float64) for f in fl] + [np.zeros(1)])
        arc_off, arc_n, t0, t1, sg, ln = [], [], [], [], [], []
        self.part_len = np.zeros((n, 2))
        for i in range(n):
            if variant == "vr" and d >= 3:
                self.part_len[i] = vr_parts(d, surfs[i], fl[i])
                arc_off.append(len(t0))
                arc_n.append(0)
                continue
            arcs = vr_arcs(d, surfs[i], fl[i], self.beta_scale[i]) if variant == "vr" else None
            if variant == "vr" and arcs is None:
                # 2D data other than a Fourier series: parts of no closed form, start by trials
                self.part_len[i] = (-1.0, -1.0)
                arc_off.append(len(t0))
                arc_n.append(0)
                continue
            arc_off.append(len(t0))
            arc_n.append(0 if arcs is None else len(arcs))
            for a, b, s_, L in (arcs or []):
                t0.append(a); t1.append(b); sg.append(s_); ln.append(L)
                self.part_len[i, 0 if s_ > 0 else 1] += L
        self.arc_off = np.array(arc_off, dtype=np.int32)
        self.arc_n = np.array(arc_n, dtype=np.int32)
        self.arc_t0 = np.array(t0 + [0.0])
        self.arc_t1 = np.array(t1 + [0.0])
        self.arc_sign = np.array(sg + [0], dtype=np.int32)
        self.arc_len = np.array(ln + [0.0])
        self.arcs = list(zip(t0, t1, sg, ln))
        self.struct = OrProblem(
            d, n, self.type.ctypes.data, self.center.ctypes.data, self.radius.ctypes.data, self.star_K.ctypes.data,
            self.star_a.ctypes.data, self.star_b.ctypes.data, self.star_s.ctypes.data, self.star_scan.ctypes.data,
            self.area.ctypes.data,
            self.is_desc.ctypes.data, self.alpha.ctypes.data, self.beta_scale.ctypes.data,
            self.thresh.ctypes.data, float(self.alpha_l1), self.flux_basis.ctypes.data, self.flux_off.ctypes.data,
            self.flux_n.ctypes.data, self.flux_coef.ctypes.data, self.arc_off.ctypes.data,
            self.arc_n.ctypes.data, self.arc_t0.ctypes.data, self.arc_t1.ctypes.data, self.arc_sign.ctypes.data,
            self.arc_len.ctypes.data, self.part_len.ctypes.data, self.ell_A.ctypes.data, self.ell_map.ctypes.data,
            self.ell_jmax.ctypes.data, self.mesh_off.ctypes.data, self.mesh_n.ctypes.data, self.tri.ctypes.data,
            self.tri_thresh.ctypes.data)


VARIANTS = {"plain": 0, "vr": 1}


def _opts(M, variant, sched_group):
    return OrOpts(int(M), VARIANTS[variant], int(sched_group))


def estimate(problem, points, n_walks, seed=0, M=None, variant="plain", sched_group=1, walk_begin=0,
             instance=0, prepared=None, point_offset=0, tile=0):
    """Algorithm 1 over every point: mean of N * (walk sum), and the standard
    error from the schedule-group means (groups of `sched_group` walkers).
    Point p uses the random stream of point id point_offset + p; with tile > 0
    (trajectories shared by a batch of points, Sec. 4.6) it uses the stream of
    id (point_offset + p) // tile, so the points of one tile see the same walks.
    Returns a dict with u [P], grad [P, d], se_u, se_grad and raw sums."""
    prep = prepared or Prepared(problem, variant)
    if tile > 0:
        parts = [estimate(problem, points[p:p + 1], n_walks, seed, M, variant, sched_group, walk_begin, instance,
                          prep, (point_offset + p) // tile) for p in range(len(points))]
        cat = {k: np.concatenate([r[k] for r in parts]) for k in ("u", "grad", "se_u", "se_grad", "sum_f",
                                                                 "sum_gm", "sum_gm2")}
        cat.update(n_walks=n_walks, n_groups=parts[0]["n_groups"] if parts else 0)
        return cat
    M = problem["M"] if M is None else M
    pts = np.ascontiguousarray(points, dtype=np.float64)
    P, d = pts.shape
    assert d == prep.dim
    sf = np.zeros((P, d + 1))
    sm = np.zeros((P, d + 1))
    sm2 = np.zeros((P, d + 1))
    G = ctypes.c_int64(0)
    o = _opts(M, variant, sched_group)
    rc = lib().or_estimate(ctypes.byref(prep.struct), ctypes.byref(o), pts.ctypes.data, P, point_offset, instance,
                           walk_begin, walk_begin + n_walks, seed, sf.ctypes.data, sm.ctypes.data,
                           sm2.ctypes.data, ctypes.byref(G))
    if rc != 0:
        raise ValueError("walk range must be a multiple of the schedule group")
    return finalize(sf, sm, sm2, n_walks, G.value)


def finalize(sf, sm, sm2, n_walks, G):
    mean = sf / n_walks
    gm = sm / G
    var = np.maximum(sm2 - G * gm * gm, 0.0) / max(G - 1, 1)
    se = np.sqrt(var / G)
    return {"u": mean[:, 0], "grad": mean[:, 1:], "se_u": se[:, 0], "se_grad": se[:, 1:],
            "sum_f": sf, "sum_gm": sm, "sum_gm2": sm2, "n_walks": n_walks, "n_groups": G}


def walks(problem, x, walk_ids, seed=0, M=None, variant="plain", sched_group=1, point_id=0, instance=0,
          prepared=None):
    """Per-walk values N * sum_i c_i Phi(x, y_i) and the gradient tally, with
    the schedule, the states, Q and T, for pathwise replay.  "scale"[:, 0] and
    [:, 1] are the walk's first-order error bounds B_u and B_g (a computation
    of the walk rounded with unit roundoff u differs by about u B from the exact
    one), [:, 2] the walk's conditioning (the largest amplification of a state
    error by consecutive line / ray steps), [:, 3] the largest ratio of the start
    flux's term magnitudes to its value; "E_y" and "E_Q" [n, 2, M+1] the error
    bounds of each state y_i and of Q_i in the same units."""
    prep = prepared or Prepared(problem, variant)
    M = problem["M"] if M is None else M
    d = prep.dim
    x = np.ascontiguousarray(x, dtype=np.float64)
    ids = np.ascontiguousarray(walk_ids, dtype=np.uint64)
    n = len(ids)
    fu = np.zeros(n)
    fg = np.zeros((n, d))
    H = np.zeros((n, M + 1), dtype=np.int32)
    Y = np.zeros((n, 2, M + 1, d))
    sc = np.zeros((n, 4))
    QT = np.zeros((n, 2, M + 1, 2))
    E = np.zeros((n, 2, M + 1, 2))
    o = _opts(M, variant, sched_group)
    lib().or_walks(ctypes.byref(prep.struct), ctypes.byref(o), x.ctypes.data, point_id, instance, ids.ctypes.data,
                   n, seed, fu.ctypes.data, fg.ctypes.data, H.ctypes.data, Y.ctypes.data, sc.ctypes.data,
                   QT.ctypes.data, E.ctypes.data)
    return {"u": fu, "grad": fg, "H": H, "Y": Y, "scale": sc, "Q": QT[..., 0], "T": QT[..., 1],
            "E_y": E[..., 0], "E_Q": E[..., 1]}


def flux_at(problem, h, y, prepared=None, tri=-1):
    prep = prepared or Prepared(problem)
    yy = np.zeros(MAX_DIM)
    yy[:prep.dim] = y
    return lib().or_test_flux(ctypes.byref(prep.struct), h, int(tri), yy.ctypes.data)


def intersections(problem, h, y, z, ray, prepared=None, exclude=-1, with_triangles=False):
    prep = prepared or Prepared(problem)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    zz = np.ascontiguousarray(z, dtype=np.float64)
    ts = np.zeros(64)
    hits = np.zeros(64, dtype=np.int32)
    q = lib().or_test_intersections(ctypes.byref(prep.struct), h, yy.ctypes.data, zz.ctypes.data, int(ray),
                                    ts.ctypes.data, int(exclude), hits.ctypes.data)
    return (ts[:q], hits[:q]) if with_triangles else ts[:q]


def real_sh(l, m, u):
    uu = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_test_real_sh(l, m, uu.ctypes.data)


def star_arclen(problem, h, t, prepared=None):
    prep = prepared or Prepared(problem)
    return lib().or_test_star_arclen(ctypes.byref(prep.struct), h, t)


def uniform_points(problem, h, n, seed=0, prepared=None, with_triangles=False):
    prep = prepared or Prepared(problem)
    out = np.zeros((n, prep.dim))
    tri = np.zeros(n, dtype=np.int32)
    t = ctypes.c_int(0)
    for w in range(n):
        y = np.zeros(prep.dim)
        lib().or_test_uniform_point(ctypes.byref(prep.struct), h, seed, 0, w, 0, y.ctypes.data, ctypes.byref(t))
        out[w] = y
        tri[w] = t.value
    return (out, tri) if with_triangles else out


def uniform_part_points(problem, h, part, n, seed=0, prepared=None):
    prep = prepared or Prepared(problem, "vr")
    out = np.zeros((n, prep.dim))
    for w in range(n):
        y = np.zeros(prep.dim)
        lib().or_test_uniform_part_point(ctypes.byref(prep.struct), h, part, seed, w, y.ctypes.data)
        out[w] = y
    return out


def directions(d, n, seed=0):
    out = np.zeros((n, d))
    for w in range(n):
        z = np.zeros(d)
        lib().or_test_direction(d, seed, w, 0, z.ctypes.data)
        out[w] = z
    return out


def threads_used():
    """Host threads the estimator over points runs on."""
    return int(lib().or_threads(0))


def set_threads(n):
    """Run the estimator over points on n host threads (n > 0); returns the count in use."""
    return int(lib().or_threads(int(n)))


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(LIB)
