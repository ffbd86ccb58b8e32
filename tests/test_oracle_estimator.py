"""The Monte Carlo oracle against exact expectations (CPU).

Each case compares the oracle's per-point estimate of u and grad u with the
exact mean of the truncated estimator (Thms 4.1-4.2): the concentric-sphere
series (2D, 3D, 6D workloads), the Nystrom series on a star with inclusions
(plain and variance-reduced, Algorithm 3), the pure Neumann problem (N = 1,
the Walk-on-Boundary special case of Sec. 2), the variance-reduced walk on
hemisphere parts in 3D and 6D, an invisible interface
(sigma_i = sigma_p, b_i = 0) and shared schedules (Algorithm 1 with W
walkers per schedule).  The test statistic is z = (estimate - exact) / SE with
the SE from the schedule-group means; with fixed seeds the outcome is
deterministic.  Planted mistakes in the oracle (Sec. 3 signs and scalings,
the range of the sign product, T in the uniform case, the normal of K*, the
truncation weight, the factor N) must be detected.
"""
import numpy as np
import pytest

from oracle import closed_form as cf
from paper_2508_16767_gb300 import workloads as wl

Z_PASS = 4.75   # Bonferroni-level bound for a few hundred z-scores
Z_CATCH = 8.0   # a planted mistake must push some |z| beyond this


def concentric_exact(prob, M, x):
    radii = [s["radius"] for s in prob["surfaces"]]
    return cf.concentric_truncated_mean(prob["dim"], radii, prob["sigma"], prob["parent"],
                                        cf.modes_from_problem(prob), M, x)


def zscores(res, u_ex, g_ex):
    zu = (res["u"] - u_ex) / res["se_u"]
    zg = (res["grad"] - g_ex) / res["se_grad"]
    return np.concatenate([zu, zg.ravel()])


def _cases():
    p1 = wl.concentric_2d_problem()
    x1 = wl.concentric_2d_points()[::5]
    p2 = wl.nested_3d_problem()
    x2 = wl.ball_points(12, 3, 12)
    p4 = wl.nested_6d_problem()
    x4 = wl.ball_points(8, 6, 14)
    # a low-conductivity inclusion (alpha_2 < 0) with its own flux jump
    p5 = wl.concentric_2d_problem()
    p5["sigma"] = [1.0, 0.25]
    p5["flux"][1] = wl.fourier([0.5, 0.0], [0.0, 0.3])
    x5 = wl.concentric_2d_points()[2::6]
    # Example 3 (3D) geometry: spheres 1 and 0.4, sigma ratio 1/2, Neumann data 5 sin(phi) cos(theta)
    p6 = {"name": "e3b", "dim": 3, "surfaces": [{"kind": "sphere", "center": [0.0] * 3, "radius": 1.0},
                                                {"kind": "sphere", "center": [0.0] * 3, "radius": 0.4}],
          "parent": [-1, 0], "sigma": [1.0, 0.5],
          "flux": [wl.real_sh({(1, 1): 5.0 * np.sqrt(4 * np.pi / 3)}, 1), wl.real_sh({(2, 0): 0.7}, 2)], "M": 6}
    x6 = wl.ball_points(10, 3, 21, radius=0.95)
    return [(p1, x1, 60000, 4), (p2, x2, 60000, 6), (p4, x4, 60000, 8), (p5, x5, 60000, 4), (p6, x6, 60000, 6)]


def _max_z(core, cases, **kw):
    zs = []
    for prob, x, W, M in cases:
        res = core.estimate(prob, x, W, seed=0, M=M, **kw)
        u_ex, g_ex = concentric_exact(prob, M, x)
        zs.append(zscores(res, u_ex, g_ex))
    return np.abs(np.concatenate(zs))


def test_concentric_workloads_match_exact_mean(oracle_core):
    z = _max_z(oracle_core, _cases())
    assert z.max() < Z_PASS
    assert 0.6 < np.sqrt(np.mean(z ** 2)) < 1.4   # SE calibration


def test_shared_schedules_same_mean(oracle_core):
    z = _max_z(oracle_core, _cases(), sched_group=32)
    assert z.max() < Z_PASS


def test_variance_reduced_concentric_2d(oracle_core):
    p1 = wl.concentric_2d_problem()
    x1 = wl.concentric_2d_points()[::3]
    res = oracle_core.estimate(p1, x1, 60000, seed=4, M=4, variant="vr")
    u_ex, g_ex = concentric_exact(p1, 4, x1)
    assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS


def test_variance_reduced_hemispheres_nd(oracle_core):
    """Algorithm 3 in d >= 3 on data linear in the unit vector (hemisphere parts,
    a zero-data interface with a dead second chain): the exact mean of the plain
    estimator, with a smaller SE than the plain walk on the same seeds."""
    p3 = wl.linear_3d_problem()
    x3 = wl.ball_points(10, 3, 31, radius=0.95)
    p6 = wl.nested_6d_problem()
    x6 = wl.ball_points(6, 6, 32)
    for prob, x, M in ((p3, x3, 6), (p6, x6, 8)):
        res = oracle_core.estimate(prob, x, 60000, seed=5, M=M, variant="vr")
        u_ex, g_ex = concentric_exact(prob, M, x)
        assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS


@pytest.mark.parametrize("dim", [4, 5])
def test_nested_4d_5d_match_exact_mean(oracle_core, dim):
    """Dimensions 4 and 5 (directions from Gaussian pairs, the d-dimensional kernels and the
    hemisphere parts of Algorithm 3): the plain and the variance-reduced estimator against
    the exact mean of the truncated estimator on two nested hyperspheres."""
    prob = wl.nested_nd_problem(dim)
    x = wl.ball_points(8, dim, 40 + dim)
    for variant, seed in (("plain", 0), ("vr", 5)):
        res = oracle_core.estimate(prob, x, 60000, seed=seed, M=8, variant=variant)
        u_ex, g_ex = concentric_exact(prob, 8, x)
        assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS, variant


def test_variance_reduced_by_trials(oracle_core):
    """Algorithm 3 where |dOmega^+/-| has no closed form (degree-2 data on 3D spheres):
    the start by 16 shared uniform trials, weighted by their fraction of each sign, has the
    plain estimator's exact mean, and a smaller SE on these workloads."""
    for prob, x in ((wl.nested_3d_problem(), wl.ball_points(10, 3, 12)),
                    (wl.zonal_3d_problem(), wl.ball_points(10, 3, 41, radius=0.95))):
        res = oracle_core.estimate(prob, x, 60000, seed=0, M=6, variant="vr")
        u_ex, g_ex = concentric_exact(prob, 6, x)
        assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS
        plain = oracle_core.estimate(prob, x, 60000, seed=0, M=6)
        assert np.sqrt(np.mean(res["se_u"] ** 2)) < 0.8 * np.sqrt(np.mean(plain["se_u"] ** 2))


def test_variance_reduced_by_trials_on_ellipsoids_and_meshes(oracle_core):
    """The start by trials on ellipsoids (Example 2, point-charge data) and on meshes (rock
    inclusions, harmonic-polynomial data), where no closed form exists: Algorithm 3's
    estimate agrees with the plain estimator's (pinned by the ellipsoid and mesh tests)
    within 4.75 combined SE, on independent seeds."""
    ell = wl.ellipsoids_problem(3)
    rocks = wl.rocks_problem(n_rocks=2, subdiv_outer=2, subdiv_rock=1, M=3)
    for prob, x, W in ((ell, wl.ellipsoid_points(ell, 6, seed=23), 40000),
                       (rocks, wl.mesh_points(rocks, 6, seed=24), 20000)):
        vr = oracle_core.estimate(prob, x, W, seed=5, variant="vr")
        plain = oracle_core.estimate(prob, x, W, seed=6)
        z = (vr["u"] - plain["u"]) / np.hypot(vr["se_u"], plain["se_u"])
        zg = (vr["grad"] - plain["grad"]) / np.hypot(vr["se_grad"], plain["se_grad"])
        assert np.abs(np.concatenate([z, zg.ravel()])).max() < Z_PASS, prob.get("name")


def test_variance_reduced_by_trials_in_2d(oracle_core):
    """2D data other than a Fourier series (harmonic-polynomial data on circles in a disk):
    the start by trials agrees with the plain estimator within 4.75 combined SE."""
    rng = np.random.default_rng(31)
    for k in range(2):
        prob = wl.manufactured_instance(2, rng, k_max=6)
        x = wl.ball_points(6, 2, 40 + k, radius=0.9)
        prep = oracle_core.Prepared(prob, "vr")
        assert np.all(prep.part_len < 0)
        vr = oracle_core.estimate(prob, x, 40000, seed=7, variant="vr", prepared=prep)
        plain = oracle_core.estimate(prob, x, 40000, seed=8)
        z = (vr["u"] - plain["u"]) / np.hypot(vr["se_u"], plain["se_u"])
        zg = (vr["grad"] - plain["grad"]) / np.hypot(vr["se_grad"], plain["se_grad"])
        assert np.abs(np.concatenate([z, zg.ravel()])).max() < Z_PASS


def test_vr_trial_weight_is_the_part_fraction(oracle_core):
    """The trial count C_k / K in the start weight Q = beta |dOmega| C_k / K: over many
    walks started on the outer sphere of the zonal case (data Y_2^0) it averages the
    exact part fractions 1 - 1/sqrt(3) and 1/sqrt(3)."""
    prob = wl.zonal_3d_problem()
    prep = oracle_core.Prepared(prob, "vr")
    assert np.all(prep.part_len < 0)                      # flagged: parts by trials
    ow = oracle_core.walks(prob, np.zeros(3), np.arange(4000, dtype=np.uint64), seed=2, M=0, variant="vr",
                           prepared=prep)
    on_outer = ow["H"][:, 0] == 0
    area = prep.area[0]
    for k, p_exact in ((0, 1 - 1 / np.sqrt(3)), (1, 1 / np.sqrt(3))):
        alive = ow["Q"][on_outer, k, 0] != 0     # no trial of that sign: the chain is dead
        y = ow["Y"][on_outer, k, 0][alive]
        beta = np.array([prep.beta_scale[0] * oracle_core.flux_at(prob, 0, yy, prepared=prep) for yy in y])
        frac = np.zeros(len(alive))
        frac[alive] = ow["Q"][on_outer, k, 0][alive] / (beta * area)
        assert np.all(np.abs(frac * 16 - np.round(frac * 16)) < 1e-9)     # a count of 16 trials
        assert np.all(np.sign(beta) == (1 if k == 0 else -1))
        assert abs(frac.mean() - p_exact) < 5 * frac.std() / np.sqrt(len(frac))


def test_vr_trial_weight_on_a_circle(oracle_core):
    """2D trial start on a circle with the harmonic-polynomial data n . grad(x_1 x_2) =
    R sin 2 theta (zero mean; its sign parts are four quarter arcs, half the circle each):
    the start weights average the part fraction 1/2, and every start lies on the circle
    in the part of its sign."""
    R = 0.8
    prob = {"dim": 2, "surfaces": [wl._sphere([0.0, 0.0], R)], "parent": [-1], "sigma": [1.0],
            "flux": [wl.harmonic_poly(1.0, [(1.0, (1, 1))], 2)], "M": 0}
    prep = oracle_core.Prepared(prob, "vr")
    assert np.all(prep.part_len < 0)
    ow = oracle_core.walks(prob, np.array([0.1, 0.2]), np.arange(3000, dtype=np.uint64), seed=4, M=0,
                           variant="vr", prepared=prep)
    for k, sgn in ((0, 1.0), (1, -1.0)):
        alive = ow["Q"][:, k, 0] != 0            # no trial of that sign (2^-16): the chain is dead
        y = ow["Y"][alive, k, 0]
        assert np.allclose(np.linalg.norm(y, axis=1), R, atol=1e-13)
        beta = np.array([prep.beta_scale[0] * oracle_core.flux_at(prob, 0, yy, prepared=prep) for yy in y])
        assert np.all(sgn * beta > 0)
        frac = np.zeros(len(alive))
        frac[alive] = ow["Q"][alive, k, 0] / (beta * prep.area[0])
        assert abs(frac.mean() - 0.5) < 5 * frac.std() / np.sqrt(len(frac))


def test_vr_trial_weight_mistake_is_detected(oracle_core):
    """A planted mistake: the trial start weighs beta by |dOmega| / 2 (as if the parts
    were halves); the zonal case's parts are not, and the exact mean catches it."""
    prob, x = wl.zonal_3d_problem(), wl.ball_points(10, 3, 41, radius=0.95)
    oracle_core.set_mutant(11)
    try:
        res = oracle_core.estimate(prob, x, 60000, seed=0, M=6, variant="vr")
    finally:
        oracle_core.set_mutant(0)
    u_ex, g_ex = concentric_exact(prob, 6, x)
    assert np.abs(zscores(res, u_ex, g_ex)).max() > Z_CATCH


def test_vr_without_reflection_is_detected(oracle_core):
    """A planted mistake: the part sampler keeps directions of the wrong sign (no
    reflection), so each chain draws from the whole sphere.  Each chain then averages
    beta |dOmega| / 2 over the whole sphere and their sum is still unbiased, so the
    exact-mean test cannot see it; the sign of the start samples does."""
    prob, x = wl.linear_3d_problem(), wl.ball_points(10, 3, 31, radius=0.95)
    prep = oracle_core.Prepared(prob, "vr")
    oracle_core.set_mutant(10)
    try:
        res = oracle_core.estimate(prob, x, 30000, seed=5, M=6, variant="vr", prepared=prep)
        y = oracle_core.uniform_part_points(prob, 0, 0, 200, seed=1, prepared=prep)
    finally:
        oracle_core.set_mutant(0)
    u_ex, g_ex = concentric_exact(prob, 6, x)
    assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS          # the mean is blind to it
    beta = np.array([oracle_core.flux_at(prob, 0, yy, prepared=prep) for yy in y])
    assert np.sum(beta < 0) > 50                                     # the sampler check is not


@pytest.mark.parametrize("variant", ["plain", "vr"])
def test_star_with_inclusions_matches_nystrom(oracle_core, variant):
    prob = wl.star_inclusions_problem(seed=3, n_incl=3)
    x = np.array([[0.1, 0.2], [-0.5, 0.3], [0.6, -0.4], [0.0, -0.7]])
    for M in (1, 3):
        res = oracle_core.estimate(prob, x, 20000, seed=1 + M, M=M, variant=variant)
        u_ex, g_ex = cf.nystrom_truncated_mean_2d(prob, M, x, n_nodes=600)
        assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS


def test_pure_neumann_disk_is_walk_on_boundary(oracle_core):
    """N = 1 (Sec. 2): Delta u = 0 in the unit disk, d_n u = cos(2 t) on the
    boundary; u = r^2 cos(2 t) / 2 up to a constant, and the estimator with
    alpha_1 = 2 is the Walk-on-Boundary estimator of Eq. WoB_neumann, exact in
    mean for every M because K* on a circle annihilates zero-mean data."""
    prob = {"dim": 2, "surfaces": [{"kind": "sphere", "center": [0.0, 0.0], "radius": 1.0}],
            "parent": [-1], "sigma": [1.0], "flux": [wl.fourier([0.0, 1.0], [0.0, 0.0])], "M": 3}
    x = wl.ball_points(10, 2, 9, radius=0.9)
    res = oracle_core.estimate(prob, x, 40000, seed=3, M=3)
    r = np.linalg.norm(x, axis=1)
    t = np.arctan2(x[:, 1], x[:, 0])
    u_ex = 0.5 * r * r * np.cos(2 * t)
    g_ex = np.stack([x[:, 0], -x[:, 1]], axis=1)
    assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS


def test_invisible_interface(oracle_core):
    """An extra surface with sigma equal to its parent's and b = 0 has
    alpha = 0 and beta = 0: the mean must not change although N and the
    schedule do."""
    prob = wl.concentric_2d_problem()
    prob2 = wl.concentric_2d_problem()
    prob2["surfaces"].append({"kind": "sphere", "center": [0.0, 0.0], "radius": 0.25})
    prob2["parent"].append(1)
    prob2["sigma"].append(prob2["sigma"][1])
    prob2["flux"].append(wl.zero_flux())
    x = wl.concentric_2d_points()[::6]
    res = oracle_core.estimate(prob2, x, 60000, seed=6, M=4)
    u_ex, g_ex = concentric_exact(prob, 4, x)
    assert np.abs(zscores(res, u_ex, g_ex)).max() < Z_PASS


@pytest.mark.parametrize("variant", ["plain", "vr"])
def test_walk_ranges_merge(oracle_core, variant):
    """Splitting the walks into ranges (resumption / sharding) and adding the
    sums reproduces the single run (the variance-reduced start by trials draws
    per walk too)."""
    prob = wl.nested_3d_problem()
    x = wl.ball_points(3, 3, 2)
    a = oracle_core.estimate(prob, x, 4096, seed=2, M=6, variant=variant)
    b1 = oracle_core.estimate(prob, x, 1024, seed=2, M=6, variant=variant)
    b2 = oracle_core.estimate(prob, x, 3072, seed=2, M=6, walk_begin=1024, variant=variant)
    assert np.allclose(a["sum_f"], b1["sum_f"] + b2["sum_f"], rtol=1e-12, atol=1e-12)
    assert np.allclose(a["sum_gm2"], b1["sum_gm2"] + b2["sum_gm2"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_planted_mistakes_are_detected(oracle_core, mutant):
    cases = _cases()
    cases = [(p, x, 30000, M) for p, x, _, M in cases]
    # short truncations make the last (half-weighted) term large
    cases += [(p, x, 30000, 1) for p, x, _, M in cases if p["dim"] in (2, 3)]
    try:
        oracle_core.set_mutant(mutant)
        z = _max_z(oracle_core, cases)
    finally:
        oracle_core.set_mutant(0)
    assert z.max() > Z_CATCH, f"planted mistake {mutant} not detected (max |z| = {z.max():.2f})"


def test_oracle_reproduces_stored_replay(oracle_core):
    """Regression: the per-walk values written by tests/golden/make_replay.py."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "replay_small.json")))
    probs = {"2d-concentric": wl.concentric_2d_problem(), "3d-nested": wl.nested_3d_problem(),
             "star-3": wl.star_inclusions_problem(seed=3, n_incl=3),
             "star-3-vr": wl.star_inclusions_problem(seed=3, n_incl=3),
             "3d-linear-vr": wl.linear_3d_problem(), "3d-zonal-vr": wl.zonal_3d_problem(),
             "4d-nested": wl.nested_nd_problem(4), "5d-nested-vr": wl.nested_nd_problem(5),
             "6d-nested": wl.nested_6d_problem(), "ellipsoids-4d": wl.ellipsoids_problem(4)}
    for c in gold["cases"]:
        r = oracle_core.walks(probs[c["name"]], np.asarray(c["x"]), np.arange(32), seed=0, M=c["M"],
                              variant=c["variant"], point_id=c["point_id"])
        assert np.array_equal(r["H"], np.asarray(c["H"]))
        assert np.allclose(r["u"], c["u"], rtol=1e-12, atol=1e-13)
        assert np.allclose(r["grad"], c["grad"], rtol=1e-12, atol=1e-13)
