"""Pins of the oracle's triangle-mesh surfaces (CPU), the paper's primary
surface representation (Sec. 5):

* line / ray intersections against the crossings of the generalised winding
  number along the line (an independent inside/outside predicate);
* uniform sampling by area: triangles are hit in proportion to their area and
  the samples satisfy int n dA = 0 and int (y - c).n dA = 3 |V| (divergence
  theorem; the volume from the signed-volume formula);
* a fine icosphere walks like the sphere it approximates: estimates agree with
  the sphere's within the O(h^2) geometric difference and the standard error.
"""
import numpy as np
import pytest
from scipy import optimize, stats

from paper_2508_16767_gb300 import workloads as wl


def rock_problem(subdiv=2, seed=3):
    V, F = wl.radial_mesh([0.1, -0.05, 0.02], 0.8, subdiv, 0.25, seed)
    return {"dim": 3, "surfaces": [wl._mesh(V, F, [0.1, -0.05, 0.02])], "parent": [-1], "sigma": [1.0],
            "flux": [wl.zero_flux()], "M": 1}, V, F


def test_mesh_intersections_match_winding_number(oracle_core):
    prob, V, F = rock_problem()
    prep = oracle_core.Prepared(prob)
    y_s, tri = oracle_core.uniform_points(prob, 0, 12, seed=4, prepared=prep, with_triangles=True)
    rng = np.random.default_rng(5)
    inside = lambda p: wl.winding_number(V, F, p) - 0.5
    for y, t0 in zip(y_s, tri):
        z = rng.standard_normal(3)
        z /= np.linalg.norm(z)
        ts, hits = oracle_core.intersections(prob, 0, y, z, False, prepared=prep, exclude=int(t0),
                                             with_triangles=True)
        grid = np.linspace(-2.5, 2.5, 2001)
        w = inside(y[None, :] + grid[:, None] * z[None, :])
        brute = []
        for j in np.nonzero(np.signbit(w[:-1]) != np.signbit(w[1:]))[0]:
            f = lambda t: float(inside((y + t * z)[None, :])[0])
            brute.append(optimize.brentq(f, grid[j], grid[j + 1], xtol=1e-12))
        brute = [t for t in brute if abs(t) > 1e-6]            # y itself is a crossing
        assert len(ts) == len(brute), (ts, brute)
        assert np.allclose(ts, brute, atol=1e-9)
        assert int(t0) not in list(hits)
        # the ray from an interior point exits an odd number of times
        p = prob["surfaces"][0]["center"]
        tr = oracle_core.intersections(prob, 0, np.asarray(p), z, True, prepared=prep)
        assert len(tr) % 2 == 1 and np.all(tr > 0)


def test_uniform_on_mesh_by_area(oracle_core):
    prob, V, F = rock_problem(subdiv=1)
    prep = oracle_core.Prepared(prob)
    y, tri = oracle_core.uniform_points(prob, 0, 30000, seed=6, prepared=prep, with_triangles=True)
    T, area = oracle_core.mesh_triangles(prob["surfaces"][0])
    # every sample lies in the plane of its triangle, inside it
    v0, e1, e2, n = T[tri, 0:3], T[tri, 3:6], T[tri, 6:9], T[tri, 9:12]
    assert np.allclose(np.einsum("ij,ij->i", y - v0, n), 0.0, atol=1e-12)
    # triangles are chosen in proportion to their area
    counts = np.bincount(tri, minlength=len(F))
    assert stats.chisquare(counts, area / area.sum() * len(y)).pvalue > 1e-3
    c = np.asarray(prob["surfaces"][0]["center"])
    vol = np.sum(np.einsum("ij,ij->i", V[F[:, 0]] - c, np.cross(V[F[:, 1]] - c, V[F[:, 2]] - c))) / 6.0
    se = lambda v: v.std() / np.sqrt(len(v))
    for k in range(3):
        assert abs(n[:, k].mean()) < 5 * se(n[:, k])
    s = np.einsum("ij,ij->i", y - c, n)
    assert abs(prep.area[0] * s.mean() - 3 * vol) < 5 * prep.area[0] * se(s)
    assert prep.area[0] == pytest.approx(area.sum(), rel=1e-14)


def test_fine_icosphere_walks_like_the_sphere(oracle_core):
    """Nested icospheres (5120 triangles each) against the nested spheres they
    approximate (same sigma, harmonic data, M = 2): u and grad u agree within
    4 combined SE plus 1 % of the data scale (the meshes differ from the
    spheres by O(h^2), about 0.3 % in area)."""
    V, F = wl.icosphere(4)
    R0, R1, c1 = 1.0, 0.45, np.array([0.2, -0.1, 0.05])
    flux = [wl.harmonic_poly(1.0, [(1.0, (1, 1, 0)), (0.5, (0, 0, 1))], 3),
            wl.harmonic_poly(-0.3, [(1.0, (1, 0, 0))], 3)]
    base = {"dim": 3, "parent": [-1, 0], "sigma": [1.0, 1.5], "flux": flux, "M": 2}
    sph = dict(base, surfaces=[wl._sphere([0, 0, 0], R0), wl._sphere(c1, R1)])
    msh = dict(base, surfaces=[wl._mesh(R0 * V, F, [0, 0, 0]), wl._mesh(c1 + R1 * V, F, c1)])
    x = np.array([[-0.4, 0.3, 0.1], [0.2, -0.1, 0.45], [0.0, -0.6, -0.2]])
    a = oracle_core.estimate(sph, x, 60000, seed=2, M=2)
    b = oracle_core.estimate(msh, x, 60000, seed=3, M=2)
    tol = 4 * np.hypot(a["se_u"], b["se_u"]) + 0.01 * np.abs(a["u"]).max()
    assert np.all(np.abs(a["u"] - b["u"]) <= tol), (a["u"], b["u"], tol)
    tol_g = 4 * np.hypot(a["se_grad"], b["se_grad"]) + 0.01 * np.abs(a["grad"]).max()
    assert np.all(np.abs(a["grad"] - b["grad"]) <= tol_g), (a["grad"], b["grad"])
