"""Deterministic expectations that pin the oracle (test infrastructure only).

1. `concentric_truncated_mean`: the exact mean of the truncated WoI estimator
   on concentric d-spheres.  By Thms 4.1-4.2 the estimator's expectation is
   sum_j S_j[gamma_j^(M)](x) with gamma^(M) = sum_{k<=M} w_k Mcal^k beta (Sec. 3,
   Eq. finite_sum_approx_ux).  On concentric spheres every operator K*_ij acts
   on a degree-l spherical harmonic as a scalar, obtained from the jump
   relation (Eq. interface_jump) and the single layer of Y_l on a sphere:
       S_R[Y_l](x) = R/(2l+d-2) (r/R)^l Y_l            (r <= R)
                   = R/(2l+d-2) (R/r)^(l+d-2) Y_l      (r >= R)
   so K*_ij = -d/dn S_j evaluated on sphere i (the average of both sides when
   i = j).  The per-mode N x N matrix power is then exact.

2. `layered_pde_solution`: the PDE of Eq. interface_problem solved directly by
   separation of variables on the same geometry (no boundary integrals): per
   mode u = (A_j r^l + B_j r^-(l+d-2)) Y_l in each layer.

3. `paper_e3a`, `paper_e3b`: the closed forms printed for Example 3 (2D
   concentric circles, Eq. C0_gradient_2D_analytical_soln; 3D concentric
   spheres, Eq. C0_gradient_3D_analytical_soln and its 3x3 system).

4. `nystrom_truncated_mean_2d`: the exact mean of the truncated estimator for
   arbitrary smooth 2D curves (off-centre circles, star curves), by the
   trapezoidal (Nystrom) discretisation of the same series:
   gamma^(M) = sum_k w_k Mcal^k beta with (K*_ij f)(x_a) = sum_b K*(x_a, y_b) f(y_b) w_b
   and the diagonal limit K*(x, x) = kappa(x) / (4 pi) on a C^2 curve.

A "mode" is a homogeneous harmonic polynomial H of degree l, given as a
callable returning (H(x), grad H(x)) for x [n, d]; on the sphere of radius R
about the origin its trace is H(y / R) = Y_l(y_hat).
"""
from __future__ import annotations

import math

import numpy as np


def omega(d):
    return 2.0 * math.pi ** (d / 2) / math.gamma(d / 2)


def alpha_beta_scale(sigma, parent):
    n = len(sigma)
    a = np.zeros(n)
    s = np.zeros(n)
    for i in range(n):
        if parent[i] < 0:
            a[i], s[i] = 2.0, 2.0 / sigma[i]
        else:
            sp, si = sigma[parent[i]], sigma[i]
            a[i], s[i] = 2.0 * (si - sp) / (sp + si), -2.0 / (sp + si)
    return a, s


def kstar_eigen(d, l, Ri, Rj):
    """Scalar action of K*_ij on Y_l, sphere i (radius Ri) receiving from sphere j."""
    den = 2 * l + d - 2
    if Ri == Rj:
        return (d - 2) / (2.0 * den)
    if Ri < Rj:
        return -l / den * (Ri / Rj) ** (l - 1)
    return (l + d - 2) / den * (Rj / Ri) ** (l + d - 1)


def truncation_weights(M):
    return np.array([1.0 - 0.5 * (k == M) for k in range(M + 1)])


def _single_layer(d, l, R, H, gH, x):
    """S_R[Y_l](x) and its gradient for Y_l = H(x_hat), H homogeneous of degree l."""
    r = np.linalg.norm(x, axis=1)
    den = 2 * l + d - 2
    inside = r <= R
    # inside:  R^(1-l)/den * H(x);  outside: R^(l+d-1)/den * r^-(2l+d-2) * H(x)
    ci = R ** (1 - l) / den
    co = R ** (l + d - 1) / den
    v = np.where(inside, ci * H, co * r ** (-den) * H)
    gi = ci * gH
    go = co * (r ** (-den))[:, None] * gH + co * H[:, None] * (-den) * (r ** (-den - 2))[:, None] * x
    g = np.where(inside[:, None], gi, go)
    return v, g


def concentric_truncated_mean(d, radii, sigma, parent, modes, M, x):
    """Exact E[u_hat_M](x), E[grad u_hat_M](x).  `modes` is a list of
    (l, fn, coef) with fn(x) -> (H, grad H) and coef[j] the amplitude of Y_l in
    b_j on sphere j (all spheres centred at the origin)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    alpha, bscale = alpha_beta_scale(sigma, parent)
    n = len(radii)
    w = truncation_weights(M)
    u = np.zeros(len(x))
    g = np.zeros_like(x)
    for l, fn, coef in modes:
        Lam = np.array([[kstar_eigen(d, l, radii[i], radii[j]) for j in range(n)] for i in range(n)])
        Mc = alpha[:, None] * Lam
        beta = bscale * np.asarray(coef, dtype=np.float64)
        gamma = np.zeros(n)
        term = beta.copy()
        for k in range(M + 1):
            gamma += w[k] * term
            term = Mc @ term
        H, gH = fn(x)
        for j in range(n):
            v, gv = _single_layer(d, l, radii[j], H, gH, x)
            u += gamma[j] * v
            g += gamma[j] * gv
    return u, g


def layered_pde_solution(d, radii, sigma, modes, x):
    """Separation-of-variables solution of Eq. interface_problem on concentric
    nested spheres R_1 > R_2 > ... (a chain: parent of j is j-1).  Per mode:
    layer j (R_{j+1} < r < R_j, sigma_j) carries (A_j + B_j r^-(2l+d-2)) H(x)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    n = len(radii)
    assert all(radii[j] > radii[j + 1] for j in range(n - 1))
    u = np.zeros(len(x))
    g = np.zeros_like(x)
    for l, fn, coef in modes:
        p = l + d - 2
        # unknowns A_0, B_0, ..., A_{n-1}, B_{n-1}; B_{n-1} = 0 (innermost region)
        m = 2 * n
        A = np.zeros((m, m))
        rhs = np.zeros(m)
        row = 0
        # radial profiles of Y_l at radius R: f(R) = A R^l + B R^-p, f'(R) = l A R^(l-1) - p B R^-(p+1)
        R = radii[0]
        A[row, 0] = sigma[0] * l * R ** (l - 1)
        A[row, 1] = -sigma[0] * p * R ** (-p - 1)
        rhs[row] = coef[0]
        row += 1
        for j in range(1, n):
            R = radii[j]
            # continuity
            A[row, 2 * (j - 1)] = R ** l
            A[row, 2 * (j - 1) + 1] = R ** (-p)
            A[row, 2 * j] = -R ** l
            A[row, 2 * j + 1] = -R ** (-p)
            row += 1
            # flux jump sigma_{j-1} du+ - sigma_j du- = b_j
            A[row, 2 * (j - 1)] = sigma[j - 1] * l * R ** (l - 1)
            A[row, 2 * (j - 1) + 1] = -sigma[j - 1] * p * R ** (-p - 1)
            A[row, 2 * j] = -sigma[j] * l * R ** (l - 1)
            A[row, 2 * j + 1] = sigma[j] * p * R ** (-p - 1)
            rhs[row] = coef[j]
            row += 1
        A[row, 2 * n - 1] = 1.0
        sol = np.linalg.solve(A, rhs)
        H, gH = fn(x)
        r = np.linalg.norm(x, axis=1)
        layer = np.zeros(len(x), dtype=int)
        for j in range(1, n):
            layer[r < radii[j]] = j
        a_c = sol[2 * layer]
        b_c = sol[2 * layer + 1]
        # u = (a r^0 + b r^-(2l+d-2)) H(x) since r^l Y = H(x) and r^-p Y = r^-(2l+d-2) H(x)
        q = 2 * l + d - 2
        fac = a_c + b_c * r ** (-q)
        u += fac * H
        g += fac[:, None] * gH + (b_c * (-q) * r ** (-q - 2) * H)[:, None] * x
    return u, g


# ---------------------------------------------------------------------------
# modes
# ---------------------------------------------------------------------------

def mode_cos2d(l):
    """H = Re (x1 + i x2)^l, trace cos(l theta) on the unit circle."""
    def fn(x):
        z = x[:, 0] + 1j * x[:, 1]
        H = (z ** l).real
        dz = l * z ** (l - 1)
        return H, np.stack([dz.real, -dz.imag], axis=1)
    return fn


def mode_sin2d(l):
    def fn(x):
        z = x[:, 0] + 1j * x[:, 1]
        H = (z ** l).imag
        dz = l * z ** (l - 1)
        return H, np.stack([dz.imag, dz.real], axis=1)
    return fn


def mode_linear(k):
    """H = x_k (degree 1 in any dimension), trace x_hat_k."""
    def fn(x):
        g = np.zeros_like(x)
        g[:, k] = 1.0
        return x[:, k].copy(), g
    return fn


def mode_real_sh(l, m):
    """r^l Y_l^m(x_hat) for the real spherical harmonics of degree <= 2
    (no Condon-Shortley phase, sin(phi) cos(theta) = sqrt(4 pi / 3) Y_1^1)."""
    c1 = math.sqrt(3 / (4 * math.pi))
    c20 = math.sqrt(5 / (16 * math.pi))
    c21 = math.sqrt(15 / (4 * math.pi))
    c22 = math.sqrt(15 / (16 * math.pi))

    def fn(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        zero = np.zeros_like(X)
        if (l, m) == (1, 1):
            return c1 * X, c1 * np.stack([1 + zero, zero, zero], 1)
        if (l, m) == (1, -1):
            return c1 * Y, c1 * np.stack([zero, 1 + zero, zero], 1)
        if (l, m) == (1, 0):
            return c1 * Z, c1 * np.stack([zero, zero, 1 + zero], 1)
        if (l, m) == (2, 0):
            return c20 * (2 * Z * Z - X * X - Y * Y), c20 * np.stack([-2 * X, -2 * Y, 4 * Z], 1)
        if (l, m) == (2, 1):
            return c21 * X * Z, c21 * np.stack([Z, zero, X], 1)
        if (l, m) == (2, -1):
            return c21 * Y * Z, c21 * np.stack([zero, Z, Y], 1)
        if (l, m) == (2, 2):
            return c22 * (X * X - Y * Y), c22 * np.stack([2 * X, -2 * Y, zero], 1)
        if (l, m) == (2, -2):
            return c21 * X * Y, c21 * np.stack([Y, X, zero], 1)
        raise ValueError((l, m))
    return fn


def modes_from_problem(problem):
    """Modes of a concentric problem built by the workload generator: Fourier
    (2D), real SH of degree <= 2 (3D) or linear harmonic polynomials."""
    d = problem["dim"]
    n = len(problem["surfaces"])
    out = {}

    def add(key, l, fn, j, v):
        if key not in out:
            out[key] = [l, fn, np.zeros(n)]
        out[key][2][j] += v

    for j, f in enumerate(problem["flux"]):
        R = problem["surfaces"][j]["radius"]
        c = f["coef"]
        if f["basis"] == "zero":
            continue
        if f["basis"] == "fourier":
            assert abs(c[0]) < 1e-14
            for k in range(1, (len(c) - 1) // 2 + 1):
                add(("c", k), k, mode_cos2d(k), j, c[2 * k - 1])
                add(("s", k), k, mode_sin2d(k), j, c[2 * k])
        elif f["basis"] == "real_sh":
            for idx, v in enumerate(c):
                if v == 0.0:
                    continue
                l = int(math.isqrt(idx))
                m = idx - l * l - l
                add(("sh", l, m), l, mode_real_sh(l, m), j, v)
        elif f["basis"] == "harmonic_poly":
            s, T = c[0], int(c[1])
            for t in range(T):
                row = c[2 + t * (d + 1): 2 + (t + 1) * (d + 1)]
                e = [int(v) for v in row[1:]]
                if sum(e) == 0:
                    continue        # a constant term of P has no gradient: no flux
                assert sum(e) == 1, "only linear harmonic polynomials have a single mode"
                k = e.index(1)
                # b = s n . grad(c x_k) = s c x_hat_k on any sphere about the origin
                add(("lin", k), 1, mode_linear(k), j, s * row[0])
        else:
            raise ValueError(f["basis"])
    return [tuple(v) for v in out.values()]


# ---------------------------------------------------------------------------
# Example 3 closed forms as printed in the paper
# ---------------------------------------------------------------------------

def paper_e3a(x, a_in=0.4, sig=1.0 / 3.0, m=3, lam=20.0):
    """u(r, t) = lam A r^m sin(m t) (r <= a), lam (B r^m + C r^-m) sin(m t)
    (a < r <= 1), A = (2/m) / (a^(2m) (sig-1) + sig + 1), B = A (sig+1)/2,
    C = B - 1/m  (Example 3, 2D)."""
    x = np.atleast_2d(x)
    r = np.linalg.norm(x, axis=1)
    t = np.arctan2(x[:, 1], x[:, 0])
    A = (2.0 / m) / (a_in ** (2 * m) * (sig - 1.0) + sig + 1.0)
    B = A * (sig + 1.0) / 2.0
    C = B - 1.0 / m
    return np.where(r <= a_in, lam * A * r ** m, lam * (B * r ** m + C * r ** (-m))) * np.sin(m * t)


def paper_e3b(x, a_in=0.4, sig=0.5, lam=5.0):
    """u = lam A r Y_1^1 (r <= a), lam (B r + C r^-2) Y_1^1 (a < r <= 1), with
    [0 1 -2; a -a -a^-2; sig -1 2a^-3] [A B C]^T = [sqrt(4 pi/3) 0 0]^T
    (Example 3, 3D)."""
    x = np.atleast_2d(x)
    M = np.array([[0.0, 1.0, -2.0], [a_in, -a_in, -a_in ** -2], [sig, -1.0, 2.0 * a_in ** -3]])
    A, B, C = np.linalg.solve(M, np.array([math.sqrt(4 * math.pi / 3), 0.0, 0.0]))
    r = np.linalg.norm(x, axis=1)
    Y11 = math.sqrt(3 / (4 * math.pi)) * x[:, 0] / r
    return np.where(r <= a_in, lam * A * r, lam * (B * r + C * r ** -2)) * Y11


# ---------------------------------------------------------------------------
# Nystrom discretisation of the truncated series for smooth 2D curves
# ---------------------------------------------------------------------------

def _curve_nodes(s, n):
    """Nodes, outward normals, speed-weighted trapezoid weights and signed
    curvature of a circle or star curve, parametrised counter-clockwise."""
    t = 2 * np.pi * np.arange(n) / n
    c = np.asarray(s["center"], dtype=np.float64)
    if s["kind"] == "sphere":
        R = s["radius"]
        r = R * np.ones(n)
        dr = np.zeros(n)
        ddr = np.zeros(n)
    else:
        R = s["radius"]
        a, b = s["star_a"], s["star_b"]
        r = R * np.ones(n)
        dr = np.zeros(n)
        ddr = np.zeros(n)
        for k in range(1, len(a)):
            r += R * (a[k] * np.cos(k * t) + b[k] * np.sin(k * t))
            dr += R * k * (-a[k] * np.sin(k * t) + b[k] * np.cos(k * t))
            ddr += -R * k * k * (a[k] * np.cos(k * t) + b[k] * np.sin(k * t))
    pts = c + np.stack([r * np.cos(t), r * np.sin(t)], 1)
    tx = dr * np.cos(t) - r * np.sin(t)
    ty = dr * np.sin(t) + r * np.cos(t)
    sp = np.hypot(tx, ty)
    nrm = np.stack([ty / sp, -tx / sp], 1)
    kappa = (r * r + 2 * dr * dr - r * ddr) / sp ** 3
    return t, pts, nrm, sp * (2 * np.pi / n), kappa


def nystrom_truncated_mean_2d(problem, M, x, n_nodes=512):
    """Exact (to quadrature accuracy) E[u_hat_M](x) and E[grad u_hat_M](x) for
    a 2D problem with circle / star surfaces and Fourier or harmonic-poly flux."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    surfs = problem["surfaces"]
    n = len(surfs)
    alpha, bscale = alpha_beta_scale(problem["sigma"], problem["parent"])
    nodes = [_curve_nodes(s, n_nodes) for s in surfs]
    beta = []
    for j, (s, f) in enumerate(zip(surfs, problem["flux"])):
        t, pts, nrm, w, kap = nodes[j]
        c = f["coef"]
        if f["basis"] == "zero":
            b = np.zeros(n_nodes)
        elif f["basis"] == "fourier":
            b = c[0] * np.ones(n_nodes)
            for k in range(1, (len(c) - 1) // 2 + 1):
                b += c[2 * k - 1] * np.cos(k * t) + c[2 * k] * np.sin(k * t)
        elif f["basis"] == "harmonic_poly":
            gP = np.zeros_like(pts)
            for i in range(int(c[1])):
                cc, e0, e1 = c[2 + i * 3], int(c[3 + i * 3]), int(c[4 + i * 3])
                if e0 > 0:
                    gP[:, 0] += cc * e0 * pts[:, 0] ** (e0 - 1) * pts[:, 1] ** e1
                if e1 > 0:
                    gP[:, 1] += cc * e1 * pts[:, 0] ** e0 * pts[:, 1] ** (e1 - 1)
            b = c[0] * np.sum(gP * nrm, axis=1)
        else:
            raise ValueError(f["basis"])
        beta.append(bscale[j] * b)
    # K*_ij blocks: K*(x_a, y_b) = (x_a - y_b) . n(x_a) / (2 pi |x_a - y_b|^2)
    K = [[None] * n for _ in range(n)]
    for i in range(n):
        _, xi, ni, _, kap = nodes[i]
        for j in range(n):
            _, yj, _, wj, _ = nodes[j]
            D = xi[:, None, :] - yj[None, :, :]
            r2 = np.sum(D * D, axis=2)
            num = np.sum(D * ni[:, None, :], axis=2)
            with np.errstate(divide="ignore", invalid="ignore"):
                Kij = num / (2 * np.pi * r2)
            if i == j:
                np.fill_diagonal(Kij, kap / (4 * np.pi))
            K[i][j] = Kij * wj[None, :]
    w = truncation_weights(M)
    gamma = [np.zeros(n_nodes) for _ in range(n)]
    term = [b.copy() for b in beta]
    for k in range(M + 1):
        for i in range(n):
            gamma[i] += w[k] * term[i]
        term = [alpha[i] * sum(K[i][j] @ term[j] for j in range(n)) for i in range(n)]
    u = np.zeros(len(x))
    g = np.zeros_like(x)
    for j in range(n):
        _, yj, _, wj, _ = nodes[j]
        D = x[:, None, :] - yj[None, :, :]
        r2 = np.sum(D * D, axis=2)
        phi = -np.log(r2) / (4 * np.pi)
        u += phi @ (gamma[j] * wj)
        g += -np.einsum("pbk,pb->pk", D, (gamma[j] * wj)[None, :] / (2 * np.pi * r2))
    return u, g
