"""The closed forms that pin the oracle, pinned in turn to the paper and to
the PDE (CPU): the truncated-series mean on concentric spheres tends, as M
grows, to (a) the separation-of-variables solution of Eq. interface_problem,
(b) the Example 3 closed forms printed in the paper, (c) the hand-derived
2D concentric solution; the layered PDE solution satisfies the interface
conditions; the Nystrom mean reproduces the concentric series."""
import json
import math
import os

import numpy as np

from oracle import closed_form as cf
from paper_2508_16767_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "example3.json")))


def _pts(d, n, seed, rmax=0.95):
    return wl.ball_points(n, d, seed, radius=rmax)


def test_e3a_series_limit_equals_paper_closed_form():
    g = GOLD["e3a_2d"]
    sig = [1.0, g["sigma_ratio"]]
    m, lam = g["m"], g["lambda"]
    # Neumann data d_r u = lam sin(m t) with sigma_1 = 1; homogeneous flux jump
    modes = [(m, cf.mode_sin2d(m), np.array([lam, 0.0]))]
    x = _pts(2, 200, 0)
    x = x[np.abs(np.linalg.norm(x, axis=1) - g["r_inner"]) > 1e-3]
    u_series, _ = cf.concentric_truncated_mean(2, [g["r_outer"], g["r_inner"]], sig, [-1, 0], modes, 80, x)
    u_paper = cf.paper_e3a(x, g["r_inner"], g["sigma_ratio"], m, lam)
    assert np.abs(u_series - u_paper).max() < 1e-10 * max(1.0, np.abs(u_paper).max())


def test_e3b_series_limit_equals_paper_closed_form():
    g = GOLD["e3b_3d"]
    sig = [1.0, g["sigma_ratio"]]
    lam = g["lambda"]
    # Neumann data lam sin(phi) cos(theta) = lam sqrt(4 pi / 3) Y_1^1
    modes = [(1, cf.mode_real_sh(1, 1), np.array([lam * math.sqrt(4 * math.pi / 3), 0.0]))]
    x = _pts(3, 200, 1)
    u_series, _ = cf.concentric_truncated_mean(3, [g["r_outer"], g["r_inner"]], sig, [-1, 0], modes, 200, x)
    u_paper = cf.paper_e3b(x, g["r_inner"], g["sigma_ratio"], lam)
    assert np.abs(u_series - u_paper).max() < 1e-9 * max(1.0, np.abs(u_paper).max())


def test_concentric_2d_closed_form():
    g = GOLD["config1_closed_form"]
    prob = wl.concentric_2d_problem()
    x = wl.concentric_2d_points()
    r = np.linalg.norm(x, axis=1)
    c = x[:, 0] / r
    u_ref = np.where(r <= 0.5, g["A"] * r * c, (g["B"] * r + g["C"] / r) * c)
    modes = cf.modes_from_problem(prob)
    u_pde, _ = cf.layered_pde_solution(2, [1.0, 0.5], prob["sigma"], modes, x)
    u_ser, _ = cf.concentric_truncated_mean(2, [1.0, 0.5], prob["sigma"], prob["parent"], modes, 60, x)
    assert np.abs(u_pde - u_ref).max() < 1e-12
    assert np.abs(u_ser - u_ref).max() < 1e-10


def _fd_check_interface_conditions(d, radii, sigma, modes):
    """sigma_1 d_n u = b_1 on the outer sphere, [u] = 0 and [sigma d_n u] = b_j on each interface."""
    rng = np.random.default_rng(3)
    for _ in range(4):
        u_hat = rng.standard_normal(d); u_hat /= np.linalg.norm(u_hat)
        for j, R in enumerate(radii):
            eps = 1e-6
            xo, xi = (R + eps) * u_hat, (R - eps) * u_hat
            fo, _ = cf.layered_pde_solution(d, radii, sigma, modes, xo[None])
            fi, _ = cf.layered_pde_solution(d, radii, sigma, modes, xi[None])
            _, go = cf.layered_pde_solution(d, radii, sigma, modes, xo[None])
            _, gi = cf.layered_pde_solution(d, radii, sigma, modes, xi[None])
            b = sum(coef[j] * fn(u_hat[None])[0][0] for l, fn, coef in modes)
            dn_in = float(gi[0] @ u_hat)
            if j == 0:
                assert abs(sigma[0] * dn_in - b) < 1e-5
            else:
                dn_out = float(go[0] @ u_hat)
                assert abs(fo[0] - fi[0]) < 1e-5
                assert abs(sigma[j - 1] * dn_out - sigma[j] * dn_in - b) < 1e-4


def test_layered_pde_solution_satisfies_interface_problem():
    p2 = wl.nested_3d_problem()
    _fd_check_interface_conditions(3, [1.0, 0.8, 0.5], p2["sigma"], cf.modes_from_problem(p2))
    p4 = wl.nested_6d_problem()
    _fd_check_interface_conditions(6, [1.0, 0.6], p4["sigma"], cf.modes_from_problem(p4))
    p1 = wl.concentric_2d_problem()
    _fd_check_interface_conditions(2, [1.0, 0.5], p1["sigma"], cf.modes_from_problem(p1))


def test_series_converges_to_pde_on_workloads():
    for prob, M in [(wl.nested_3d_problem(), 120), (wl.nested_6d_problem(), 120), (wl.concentric_2d_problem(), 60)]:
        d = prob["dim"]
        radii = [s["radius"] for s in prob["surfaces"]]
        modes = cf.modes_from_problem(prob)
        x = _pts(d, 100, 7)
        ok = np.min(np.abs(np.linalg.norm(x, axis=1)[:, None] - np.asarray(radii)[None]), axis=1) > 1e-3
        x = x[ok]
        u_s, g_s = cf.concentric_truncated_mean(d, radii, prob["sigma"], prob["parent"], modes, M, x)
        u_p, g_p = cf.layered_pde_solution(d, radii, prob["sigma"], modes, x)
        assert np.abs(u_s - u_p).max() < 1e-8
        assert np.abs(g_s - g_p).max() < 1e-7


def test_nystrom_reproduces_concentric_series():
    prob = wl.concentric_2d_problem()
    prob["flux"][1] = wl.fourier([0.5, 0.2], [0.0, -0.4])
    x = np.array([[0.1, 0.2], [0.3, -0.6], [-0.7, 0.1], [0.05, -0.2]])
    modes = cf.modes_from_problem(prob)
    for M in [0, 1, 3, 6]:
        u_a, g_a = cf.concentric_truncated_mean(2, [1.0, 0.5], prob["sigma"], prob["parent"], modes, M, x)
        u_n, g_n = cf.nystrom_truncated_mean_2d(prob, M, x, n_nodes=256)
        assert np.abs(u_a - u_n).max() < 1e-11
        assert np.abs(g_a - g_n).max() < 1e-10


def test_nystrom_converges_on_star():
    prob = wl.star_inclusions_problem(seed=3, n_incl=3)
    x = np.array([[0.1, 0.2], [-0.5, 0.3], [0.6, -0.4]])
    u1, g1 = cf.nystrom_truncated_mean_2d(prob, 3, x, n_nodes=600)
    u2, g2 = cf.nystrom_truncated_mean_2d(prob, 3, x, n_nodes=1000)
    assert np.abs(u1 - u2).max() < 1e-12
    assert np.abs(g1 - g2).max() < 1e-11
