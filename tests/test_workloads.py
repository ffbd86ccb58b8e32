"""The synthetic workloads satisfy the problem's hypotheses (Sec. 1): properly
nested, non-overlapping surfaces; flux data with zero mean on every surface
(the compatibility condition of Eq. interface_problem), hence also the total
balance; harmonic manufactured solutions; evaluation points inside Omega."""
import math

import numpy as np

from paper_2508_16767_gb300 import workloads as wl


def surface_integral_2d(s, f, n=8192):
    t = 2 * np.pi * np.arange(n) / n
    c = np.asarray(s["center"])
    if s["kind"] == "sphere":
        r = s["radius"] * np.ones(n); dr = np.zeros(n)
    else:
        a, b = s["star_a"], s["star_b"]
        r = s["radius"] * (1 + sum(a[k] * np.cos(k * t) + b[k] * np.sin(k * t) for k in range(1, len(a))))
        dr = s["radius"] * sum(k * (-a[k] * np.sin(k * t) + b[k] * np.cos(k * t)) for k in range(1, len(a)))
    pts = c + np.stack([r * np.cos(t), r * np.sin(t)], 1)
    tx = dr * np.cos(t) - r * np.sin(t); ty = dr * np.sin(t) + r * np.cos(t)
    sp = np.hypot(tx, ty)
    nrm = np.stack([ty / sp, -tx / sp], 1)
    vals = f(pts, nrm, t)
    return float(np.sum(vals * sp) * 2 * np.pi / n), float(np.sum(np.abs(vals) * sp) * 2 * np.pi / n)


def fourier_vals(coef):
    def f(pts, nrm, t):
        v = coef[0] * np.ones_like(t)
        for k in range(1, (len(coef) - 1) // 2 + 1):
            v = v + coef[2 * k - 1] * np.cos(k * t) + coef[2 * k] * np.sin(k * t)
        return v
    return f


def test_star_workload_compatibility_and_layout():
    prob = wl.star_inclusions_problem()
    surfs = prob["surfaces"]
    assert len(surfs) == 33 and prob["parent"] == [-1] + [0] * 32
    total = 0.0
    for s, fl in zip(surfs, prob["flux"]):
        integ, l1 = surface_integral_2d(s, fourier_vals(fl["coef"]))
        assert abs(integ) < 1e-10 * max(l1, 1.0)
        total += integ
    assert abs(total) < 1e-9
    # inclusions: inside the star, gap >= 0.02 to each other and to the star
    t = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    a = surfs[0]["star_a"]
    r = 1 + a[5] * np.cos(5 * t)
    curve = np.stack([r * np.cos(t), r * np.sin(t)], 1)
    for i, s in enumerate(surfs[1:]):
        c = np.asarray(s["center"])
        assert 0.03 <= s["radius"] <= 0.08
        assert np.min(np.linalg.norm(curve - c, axis=1)) >= s["radius"] + 0.02 - 1e-9
        for s2 in surfs[1 + i + 1:]:
            assert np.linalg.norm(c - np.asarray(s2["center"])) >= s["radius"] + s2["radius"] + 0.02 - 1e-12
    sig = np.asarray(prob["sigma"][1:])
    assert np.all((sig >= 0.1) & (sig <= 10.0))


def test_star_points_recipe():
    prob = wl.star_inclusions_problem()
    x = wl.star_inclusions_points(prob, 2000)
    th = np.arctan2(x[:, 1], x[:, 0])
    a = prob["surfaces"][0]["star_a"]
    assert np.all(np.linalg.norm(x, axis=1) < 1 + a[5] * np.cos(5 * th))
    # distance to the nearest surface: about 30% within 0.01
    t = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    r = 1 + a[5] * np.cos(5 * t)
    curve = np.stack([r * np.cos(t), r * np.sin(t)], 1)
    dmin = np.min(np.linalg.norm(x[:, None, :] - curve[None, ::4, :], axis=2), axis=1)
    for s in prob["surfaces"][1:]:
        dmin = np.minimum(dmin, np.abs(np.linalg.norm(x - np.asarray(s["center"]), axis=1) - s["radius"]))
    frac = np.mean(dmin <= 0.0105)
    assert 0.28 <= frac <= 0.40


def test_layered_workloads():
    p1 = wl.concentric_2d_problem()
    for s, fl in zip(p1["surfaces"], p1["flux"]):
        integ, _ = surface_integral_2d(s, fourier_vals(fl["coef"]))
        assert abs(integ) < 1e-12
    assert len(wl.concentric_2d_points()) == 64
    p2 = wl.nested_3d_problem()
    for fl in p2["flux"]:
        assert fl["coef"][0] == 0.0          # no l = 0 term: zero mean on a sphere
    x = wl.ball_points(4096, 3, 12)
    assert x.shape == (4096, 3) and np.all(np.linalg.norm(x, axis=1) < 1)
    p4 = wl.nested_6d_problem()
    assert p4["dim"] == 6 and p4["sigma"] == [1.0, 4.0]


def laplacian_of_poly(terms, d):
    out = {}
    for c, e in terms:
        for k in range(d):
            if e[k] >= 2:
                ee = list(e); ee[k] -= 2
                out[tuple(ee)] = out.get(tuple(ee), 0.0) + c * e[k] * (e[k] - 1)
    return out


def test_batch_instances_are_valid_manufactured_problems():
    inst = wl.batch_instances(n_inst=16, k_max=64, p_range=(16, 64), w_range=(1e4, 1e5))
    for it in inst:
        prob = it["problem"]
        d = prob["dim"]
        lap = laplacian_of_poly(prob["u_h"], d)
        assert all(abs(v) < 1e-12 for v in lap.values())       # u_h harmonic => compatible data
        cs = [np.asarray(s["center"]) for s in prob["surfaces"][1:]]
        rs = [s["radius"] for s in prob["surfaces"][1:]]
        for i in range(len(cs)):
            assert np.linalg.norm(cs[i]) + rs[i] < 1.0
            for j in range(i + 1, len(cs)):
                assert np.linalg.norm(cs[i] - cs[j]) > rs[i] + rs[j]
        assert 16 <= len(it["points"]) <= 64
        assert it["n_walks"] % 32 == 0 and 1e4 - 32 <= it["n_walks"] <= 1e5 + 32
        # the flux is sigma_1 dn u_h on the boundary and (sigma_p - sigma_i) dn u_h on interfaces
        assert prob["flux"][0]["coef"][0] == prob["sigma"][0]
        for i in range(1, len(prob["surfaces"])):
            assert math.isclose(prob["flux"][i]["coef"][0], prob["sigma"][0] - prob["sigma"][i])
