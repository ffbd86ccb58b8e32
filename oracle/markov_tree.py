"""The naive Walk-on-Interfaces estimator on its Markov tree (Sec. 4.2,
Eq. naive_woi_estimator, Sec. 4.2.3 "Reuse of Markov Chains"), for M = 1.

TEST INFRASTRUCTURE ONLY: an independent cross-check of the scheduled WoI
estimator of the C oracle (Thm 4.2).  It shares nothing with it but the problem
dictionary: its own numpy random numbers, its own geometry (circles and
d-spheres), its own alpha / beta scaling and no schedule at all.

For M = 1 the truncated series (Sec. 3, weights w_0 = 1, w_1 = 1/2) is

    u(x) ~ sum_{h0} E[Q_(h0) Phi(x, Y_(h0))]
           + 1/2 sum_{h0, h1} alpha_{h1} E[Q_(h1,h0) T_(h1,h0) Phi(x, Y_(h1,h0))],

and one observation walks the whole tree: a uniform point y_(h0) on every
surface (Q = beta(y) |dOmega_h0|, Eq. naive_woi_p0), then from each of them one
transition to every surface h1 (Eqs. naive_woi_p, naive_woi_Q, naive_woi_T):
the other end of an isotropic line if h1 = h0 (Q *= 1/2), the exit of an
isotropic ray if h0 is a descendant of h1, a uniform point with
Q *= K*(y_(h1,h0), y_(h0)) |dOmega_h1| otherwise.
"""
from __future__ import annotations

import math

import numpy as np


def _omega(d):
    return 2.0 * math.pi ** (d / 2) / math.gamma(d / 2)


def _phi(d, x, y):
    r = np.linalg.norm(y - x[None, :], axis=1)
    if d == 2:
        return -np.log(r) / (2 * math.pi)
    return r ** (2 - d) / ((d - 2) * _omega(d))


def _unit(rng, n, d):
    g = rng.standard_normal((n, d))
    return g / np.linalg.norm(g, axis=1)[:, None]


def _flux(problem, h, y):
    """b_h at points y [n, d] for the Fourier (2D), harmonic-polynomial and
    point-charge data of the problem dictionary."""
    d = problem["dim"]
    s = problem["surfaces"][h]
    f = problem["flux"][h]
    c = np.asarray(s["center"], dtype=np.float64)
    n = (y - c) / s["radius"]
    coef = np.asarray(f["coef"], dtype=np.float64)
    if f["basis"] == "zero":
        return np.zeros(len(y))
    if f["basis"] == "fourier":
        t = np.arctan2(n[:, 1], n[:, 0])
        v = np.full(len(y), coef[0])
        for k in range(1, (len(coef) - 1) // 2 + 1):
            v += coef[2 * k - 1] * np.cos(k * t) + coef[2 * k] * np.sin(k * t)
        return v
    if f["basis"] == "harmonic_poly":
        sc, T = coef[0], int(coef[1])
        grad = np.zeros_like(y)
        for t in range(T):
            row = coef[2 + t * (d + 1): 2 + (t + 1) * (d + 1)]
            e = row[1:].astype(int)
            for k in range(d):
                if e[k] == 0:
                    continue
                ee = e.copy()
                ee[k] -= 1
                grad[:, k] += row[0] * e[k] * np.prod(y ** ee[None, :], axis=1)
        return sc * np.sum(n * grad, axis=1)
    if f["basis"] == "point_charge":
        x0 = coef[1:]
        e = y - x0
        r = np.linalg.norm(e, axis=1)
        return coef[0] * (2 - d) * r ** (-d) * np.sum(e * n, axis=1)
    raise ValueError(f["basis"])


def _descendant(parent, a, b):
    p = parent[a]
    while p >= 0:
        if p == b:
            return True
        p = parent[p]
    return False


def estimate_m1(problem, x, n_trees, seed=0):
    """Mean and standard error of the M = 1 naive estimator at x (spheres only)."""
    d = int(problem["dim"])
    surfs = problem["surfaces"]
    N = len(surfs)
    assert all(s["kind"] == "sphere" for s in surfs)
    parent = [int(p) for p in problem["parent"]]
    sigma = [float(v) for v in problem["sigma"]]
    alpha = [2.0 if parent[i] < 0 else 2.0 * (sigma[i] - sigma[parent[i]]) / (sigma[parent[i]] + sigma[i])
             for i in range(N)]
    bscale = [2.0 / sigma[0] if parent[i] < 0 else -2.0 / (sigma[parent[i]] + sigma[i]) for i in range(N)]
    R = [float(s["radius"]) for s in surfs]
    C = [np.asarray(s["center"], dtype=np.float64) for s in surfs]
    area = [_omega(d) * r ** (d - 1) for r in R]
    rng = np.random.default_rng(seed)
    x = np.asarray(x, dtype=np.float64)
    total = np.zeros(n_trees)
    for h0 in range(N):
        y0 = C[h0] + R[h0] * _unit(rng, n_trees, d)
        Q0 = bscale[h0] * _flux(problem, h0, y0) * area[h0]
        total += Q0 * _phi(d, x, y0)
        for h1 in range(N):
            z = _unit(rng, n_trees, d)
            dy = y0 - C[h1]
            b = np.sum(z * dy, axis=1)
            if h1 == h0:
                # the other end of the chord: t = -2 b; Q *= 1/2; T *= q sign = +1
                y1 = y0 - 2 * b[:, None] * z
                Q1 = 0.5 * Q0
                T1 = np.ones(n_trees)
            elif _descendant(parent, h0, h1):
                # ray from inside the sphere h1: the positive root; T *= q sign = +1
                c0 = np.sum(dy * dy, axis=1) - R[h1] ** 2
                t = -b + np.sqrt(b * b - c0)
                y1 = y0 + t[:, None] * z
                Q1 = Q0.copy()
                T1 = np.ones(n_trees)
            else:
                # uniform on sphere h1: Q *= K*(y1, y0) |dOmega_h1| with the normal at y1
                y1 = C[h1] + R[h1] * z
                diff = y1 - y0
                r = np.linalg.norm(diff, axis=1)
                kstar = np.sum(diff * z, axis=1) / (_omega(d) * r ** d)
                Q1 = Q0 * kstar * area[h1]
                T1 = np.ones(n_trees)
            total += 0.5 * alpha[h1] * Q1 * T1 * _phi(d, x, y1)
    return float(total.mean()), float(total.std(ddof=1) / math.sqrt(n_trees))
