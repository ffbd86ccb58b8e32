"""Pins of the oracle's per-walk error bound (the tolerance scale of the replay tests).

The replay tests compare the library's walks with the oracle's walk by walk, to
1e-12 (FP64) and 1e-5 (FP32) of the bound B the oracle computes along each walk:
the first-order change of the tallies when every state, the evaluation point and
every factor carry a relative error of one unit roundoff (see the error-bound
comment in woi_oracle.c).  Here the bound is checked against a direct experiment,
so that it is not only the oracle's word:

* every walk state y (on surface s) is moved by rel |y - c_s| and the evaluation
  point by rel |x - c_s| in each tally; the tallies then change by at most
  rel B (about 0.2-1 rel B at the worst walk: the bound is attained within a
  small factor, it is not vacuous), on every surface family and variant, and at
  evaluation points 1e-2 ... 1e-5 from an interface (the near-interface regime,
  where Phi and grad Phi are steep in the states);
* a bound without its states' term (a plausible mistake) fails the same
  experiment near an interface;
* the amplification of a state error by a line or ray step whose crossing is a
  root (star curves, meshes, rays), 1 + 1 / |n(y') . z|, against the crossing of
  the perturbed line, and its absence for a chord of a sphere or ellipsoid, which
  the oracle takes as the reflection t = -2 b (Sec. 2: the intersections of the
  line through y_{i-1} other than y_{i-1}).
"""
import numpy as np
import pytest

from paper_2508_16767_gb300 import workloads as wl

REL = 1e-11


@pytest.fixture(scope="module")
def O(oracle_core):
    yield oracle_core
    oracle_core.set_perturb(0.0)
    oracle_core.set_mutant_bound(0)


def _problems():
    rocks = wl.rocks_problem(n_rocks=3, subdiv_outer=3, subdiv_rock=2, M=4)
    star3 = wl.star_inclusions_problem(seed=3, n_incl=3)
    star32 = wl.star_inclusions_problem()
    return {
        "2d-concentric": (wl.concentric_2d_problem(), "plain"),
        "2d-concentric-vr": (wl.concentric_2d_problem(), "vr"),
        "3d-nested": (wl.nested_3d_problem(), "plain"),
        "3d-nested-vr": (wl.nested_3d_problem(), "vr"),
        "6d-nested": (wl.nested_6d_problem(), "plain"),
        "star-3": (star3, "plain"),
        "star-32-vr": (star32, "vr"),
        "mesh-rocks": (rocks, "plain"),
        "ellipsoids-3d": (wl.ellipsoids_problem(3), "plain"),
    }


def _points(name, prob):
    if name.startswith("star"):
        return np.array([[0.1, 0.2], [-0.5, 0.3]])
    if name.startswith("mesh"):
        return wl.mesh_points(prob, 2, seed=61)
    if name.startswith("ellipsoids"):
        return wl.ellipsoid_points(prob, 2, seed=53)
    return wl.ball_points(2, prob["dim"], 5, radius=0.9)


def _near_cases():
    """(name, problem, point, delta): points at normal distance delta from an interface."""
    out = []
    deltas = [1e-2, 1e-3, 1e-4, 1e-5]
    for name, prob, i, side in [("3d-nested", wl.nested_3d_problem(), 1, -1), ("3d-nested", wl.nested_3d_problem(), 2, 1),
                                ("2d-concentric", wl.concentric_2d_problem(), 1, 1),
                                ("star-32", wl.star_inclusions_problem(), 0, -1),
                                ("star-32", wl.star_inclusions_problem(), 3, 1)]:
        for dl, x in zip(deltas, wl.near_surface_points(prob, i, deltas, side, seed=5)):
            out.append((f"{name}-s{i}{'+' if side > 0 else '-'}{dl:.0e}", prob, x, dl))
    return out


def _response(O, prob, x, variant, n=2000, mutant_bound=0):
    """Change of each walk's tallies under the perturbation, in units of rel B."""
    ids = np.arange(n, dtype=np.uint64)
    O.set_mutant_bound(mutant_bound)
    try:
        b = O.walks(prob, x, ids, seed=7, M=prob["M"], variant=variant)
        O.set_perturb(REL)
        p = O.walks(prob, x, ids, seed=7, M=prob["M"], variant=variant)
    finally:
        O.set_perturb(0.0)
        O.set_mutant_bound(0)
    same = np.all(b["H"] == p["H"], axis=1) & np.all(b["T"] == p["T"], axis=(1, 2))
    du = np.abs(p["u"] - b["u"])
    dg = np.max(np.abs(p["grad"] - b["grad"]), axis=1)
    ru = np.where(du > 0, du / np.maximum(REL * b["scale"][:, 0], 1e-300), 0.0)
    rg = np.where(dg > 0, dg / np.maximum(REL * b["scale"][:, 1], 1e-300), 0.0)
    return ru[same], rg[same], int(np.sum(~same))


@pytest.mark.parametrize("name", list(_problems()))
def test_bound_covers_perturbed_walks(O, name):
    prob, variant = _problems()[name]
    for x in _points(name, prob):
        ru, rg, flips = _response(O, prob, x, variant)
        assert flips == 0, (name, flips)         # a 1e-11 move changes no discrete decision here
        assert ru.max() <= 1.5 and rg.max() <= 1.5, (name, ru.max(), rg.max())
        assert max(ru.max(), rg.max()) >= 0.05, (name, ru.max(), rg.max())   # attained, not vacuous


@pytest.mark.parametrize("case", _near_cases(), ids=[c[0] for c in _near_cases()])
def test_bound_covers_near_interface_points(O, case):
    name, prob, x, delta = case
    ru, rg, flips = _response(O, prob, x, "plain")
    assert flips == 0
    assert ru.max() <= 1.5 and rg.max() <= 1.5, (name, ru.max(), rg.max())
    assert max(ru.max(), rg.max()) >= 0.1, (name, ru.max(), rg.max())


def test_bound_without_states_term_is_caught(O):
    """Planted mistake: the bound without the sensitivity of Phi and grad Phi to the
    states and to x fails the perturbation near an interface."""
    worst = 0.0
    for name, prob, x, delta in _near_cases():
        ru, rg, _ = _response(O, prob, x, "plain", n=1000, mutant_bound=1)
        worst = max(worst, ru.max(), rg.max())
    assert worst > 5.0, worst


# ---------------------------------------------------------------------------
# the amplification factor of one line / ray step
# ---------------------------------------------------------------------------

def _star_normal(s, y):
    from oracle.core import star_r
    c = np.asarray(s["center"])
    t = np.arctan2(y[1] - c[1], y[0] - c[0])
    r, dr = star_r(s, t)
    tx, ty = dr * np.cos(t) - r * np.sin(t), dr * np.sin(t) + r * np.cos(t)
    n = np.array([ty, -tx])
    return n / np.linalg.norm(n)


def _crossing_shift(O, prob, prep, h, y, z, ray, exclude, t_ref, n_start, eps):
    """Move of the crossing nearest to parameter t_ref when y moves by eps n_start."""
    ts = O.intersections(prob, h, y + eps * n_start, z, ray, prepared=prep, exclude=exclude)
    t2 = ts[np.argmin(np.abs(ts - t_ref))]
    return np.linalg.norm((y + eps * n_start + t2 * z) - (y + t_ref * z)) / eps


def test_star_chord_amplification(O):
    """Near-tangent chords of the star: a start moved by eps off the curve moves the other
    crossing by about eps / |n(y') . z| (and never by more than eps (1 + 1 / |n(y') . z|))."""
    prob = wl.star_inclusions_problem(seed=3, n_incl=3)
    s = prob["surfaces"][0]
    prep = O.Prepared(prob)
    ys = O.uniform_points(prob, 0, 40, seed=2, prepared=prep)
    rng = np.random.default_rng(1)
    attained = []
    for y in ys:
        n = _star_normal(s, y)
        tang = np.array([-n[1], n[0]])
        for phi in (1e-1, 1e-2, 1e-3):
            a = phi * rng.choice([-1, 1])
            z = np.cos(a) * tang + np.sin(a) * n
            ts = O.intersections(prob, 0, y, z, 0, prepared=prep)
            if len(ts) == 0:
                continue
            t = ts[np.argmin(np.abs(ts))]
            yn = y + t * z
            nz = abs(np.dot(_star_normal(s, yn), z))
            amp = 1.0 + 1.0 / nz
            shift = _crossing_shift(O, prob, prep, 0, y, z, 0, -1, t, n, 1e-11)
            assert shift <= 1.05 * amp, (shift, amp)
            if amp > 30:
                attained.append(shift / (amp - 1.0))
    assert len(attained) > 10 and np.median(attained) > 0.5, attained


def test_mesh_line_amplification(O):
    prob = wl.rocks_problem(n_rocks=3, subdiv_outer=3, subdiv_rock=2, M=4)
    prep = O.Prepared(prob)
    ys, tris = O.uniform_points(prob, 0, 300, seed=3, prepared=prep, with_triangles=True)
    zs = O.directions(3, 300, seed=4)
    normals = prep.tri[:, 9:12]
    ratios = []
    for y, j, z in zip(ys, tris, zs):
        ts, hit = O.intersections(prob, 0, y, z, 0, prepared=prep, exclude=int(j), with_triangles=True)
        for t, tj in zip(ts, hit):
            nz = abs(np.dot(normals[tj], z))
            amp = 1.0 + 1.0 / nz
            shift = _crossing_shift(O, prob, prep, 0, y, z, 0, int(j), t, normals[j], 1e-11)
            assert shift <= 1.05 * amp, (shift, amp)
            ratios.append(shift / amp)
    assert max(ratios) > 0.5


def test_sphere_chords_are_not_amplified_and_rays_are_bounded(O):
    """A chord of a circle / sphere / ellipsoid is the reflection t = -2 b: the other end
    moves with the start, however close to tangent the chord is.  A ray from an inner
    sphere to the outer one meets it at |n . z| >= sqrt(1 - (r_in / R)^2)."""
    for prob, h in [(wl.concentric_2d_problem(), 1), (wl.nested_3d_problem(), 1), (wl.ellipsoids_problem(3), 0)]:
        prep = O.Prepared(prob)
        d = prob["dim"]
        ys = O.uniform_points(prob, h, 30, seed=6, prepared=prep)
        c = np.asarray(prob["surfaces"][h]["center"])
        for y in ys:
            if prob["surfaces"][h]["kind"] == "sphere":
                n = (y - c) / np.linalg.norm(y - c)
            else:
                A = np.asarray(prob["surfaces"][h]["matrix"])
                n = A @ (y - c)
                n /= np.linalg.norm(n)
            t0 = np.zeros(d)
            t0[0] = 1.0
            tang = t0 - np.dot(t0, n) * n
            tang /= np.linalg.norm(tang)
            for phi in (1e-2, 1e-4, 1e-6):
                z = np.cos(phi) * tang + np.sin(phi) * n
                ts = O.intersections(prob, h, y, z, 0, prepared=prep)
                assert len(ts) == 1
                shift = _crossing_shift(O, prob, prep, h, y, z, 0, -1, ts[0], n, 1e-11)
                assert shift <= 2.5, (shift, phi)
    prob = wl.nested_3d_problem()
    prep = O.Prepared(prob)
    ys = O.uniform_points(prob, 1, 50, seed=8, prepared=prep)
    zs = O.directions(3, 50, seed=9)
    bound = 1.0 + 1.0 / np.sqrt(1.0 - 0.8 ** 2)
    for y, z in zip(ys, zs):
        ts = O.intersections(prob, 0, y, z, 1, prepared=prep)
        assert len(ts) == 1
        n = y / np.linalg.norm(y)
        assert _crossing_shift(O, prob, prep, 0, y, z, 1, -1, ts[0], n, 1e-11) <= 1.05 * bound
