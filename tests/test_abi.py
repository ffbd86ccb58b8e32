"""The C-ABI library loads, exports every entry point that include/woi.h
declares, and rejects bad input on the host (no GPU needed: no kernel runs)."""
import os
import re

import numpy as np
import pytest

from paper_2508_16767_gb300 import build as B
from paper_2508_16767_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def woi():
    B.build()
    from paper_2508_16767_gb300 import woi as W
    return W


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "woi.h")).read()
    return sorted(set(re.findall(r"WOI_API\s+[\w\s\*]*?\b(woi_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(woi):
    names = declared_entry_points()
    assert len(names) >= 10
    for n in names:
        assert hasattr(woi.lib, n), n
    assert set(names) == set(woi.EXPORTED)
    assert "sm_103a" in woi.version()


def test_geometry_validation(woi):
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(7, [wl._sphere([0] * 6, 1.0)], [-1])
    assert e.value.status == 1
    # overlapping inclusions
    surfs = [wl._sphere([0, 0], 1.0), wl._sphere([0.2, 0], 0.3), wl._sphere([-0.2, 0], 0.3)]
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(2, surfs, [-1, 0, 0])
    assert e.value.status == 2
    # inclusion poking out of its parent
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(2, [wl._sphere([0, 0], 1.0), wl._sphere([0.8, 0], 0.3)], [-1, 0])
    assert e.value.status == 2
    # parent cycle
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(2, [wl._sphere([0, 0], 1.0), wl._sphere([0, 0], 0.5), wl._sphere([0, 0], 0.2)],
                                [-1, 2, 1])
    assert e.value.status == 1
    # star in 3D
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(3, [wl._star([0, 0, 0], 1.0, [0, 0.1], [0, 0])], [-1])
    assert e.value.status == 4
    # circle crossing a star boundary
    a = [0, 0, 0, 0, 0, 0.15]
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(2, [wl._star([0, 0], 1.0, a, [0] * 6), wl._sphere([1.05, 0], 0.15)], [-1, 0])
    assert e.value.status == 2
    # the star workload is valid
    prob = wl.star_inclusions_problem()
    h = woi.Geometry(prob)
    h.close()


def test_data_validation(woi):
    prob = wl.concentric_2d_problem()
    h = woi.woi_create_geometry(2, prob["surfaces"], prob["parent"])
    try:
        bad = [wl.fourier([1.0], [0.0], a0=0.3), prob["flux"][1]]       # non-zero mean on dOmega_1
        with pytest.raises(woi.WoiError) as e:
            woi.woi_set_sigma_and_data(h, prob["sigma"], bad)
        assert e.value.status == 3
        with pytest.raises(woi.WoiError) as e:
            woi.woi_set_sigma_and_data(h, [0.0, 2.0], prob["flux"])
        assert e.value.status == 1
        nonharm = [wl.harmonic_poly(1.0, [(1.0, (2, 0))], 2), prob["flux"][1]]   # P = x^2 is not harmonic
        with pytest.raises(woi.WoiError) as e:
            woi.woi_set_sigma_and_data(h, prob["sigma"], nonharm)
        assert e.value.status == 3
        with pytest.raises(woi.WoiError) as e:
            woi.woi_set_sigma_and_data(h, prob["sigma"], [wl.real_sh({(1, 0): 1.0}, 1), prob["flux"][1]])
        assert e.value.status == 4
        woi.woi_set_sigma_and_data(h, prob["sigma"], prob["flux"])
    finally:
        woi.lib.woi_destroy_geometry(h)


def test_estimate_argument_checks_and_no_device(woi):
    """Option checks come first; without a GPU the call reports WOI_E_NO_DEVICE."""
    g = woi.Geometry(wl.nested_3d_problem())
    pts = wl.ball_points(4, 3, 1)
    with pytest.raises(woi.WoiError) as e:
        woi.woi_estimate(g, pts, 1000, sched_group=32)           # 1000 is not a multiple of 32
    assert e.value.status == 1
    with pytest.raises(woi.WoiError) as e:
        woi.woi_estimate(g, pts, 1024, M=40)
    assert e.value.status == 1
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(woi.WoiError) as e:
            woi.woi_estimate(g, pts, 1024)
        assert e.value.status == 5
        # the variance-reduced walk passes the option checks everywhere (2D arcs or trials,
        # d >= 3 hemispheres or trials) on circles, spheres, ellipsoids and meshes: only the
        # missing device stops it
        ell = wl.ellipsoids_problem(3)
        rocks = wl.rocks_problem(n_rocks=1, subdiv_outer=1, subdiv_rock=1, M=3)
        man2 = wl.manufactured_instance(2, np.random.default_rng(3), k_max=4)
        for prob, x in ((man2, wl.ball_points(4, 2, 1, radius=0.5)),
                        (wl.nested_3d_problem(), pts), (wl.linear_3d_problem(), pts),
                        (wl.nested_6d_problem(), wl.ball_points(4, 6, 1)),
                        (ell, wl.ellipsoid_points(ell, 4, seed=1)), (rocks, wl.mesh_points(rocks, 4, seed=1))):
            gv = woi.Geometry(prob)
            with pytest.raises(woi.WoiError) as e:
                woi.woi_estimate(gv, x, 1024, variant="vr")
            assert e.value.status == 5, prob.get("name")
            gv.close()
    g.close()


def test_ellipsoid_host_geometry(woi):
    """Ellipsoids (Example 2) on the host side of the library: the area the
    estimator uses equals the oracle's (an independent quadrature of the same
    formula, scipy instead of Gauss-Legendre; eigenvectors from numpy instead of
    Jacobi), the printed Example 2 geometry is rejected as not nested, and bad
    matrices and charges inside a surface are rejected."""
    from oracle import core
    for d in (3, 4, 5, 6):
        prob = wl.ellipsoids_problem(d)
        prep = core.Prepared(prob)
        with woi.Geometry(prob) as g:
            for i in range(3):
                assert g.surface_area(i) == pytest.approx(prep.area[i], rel=1e-11)
    # a strongly eccentric rotated ellipsoid
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((4, 4)))
    A = Q @ np.diag([0.5, 2.0, 30.0, 400.0]) @ Q.T
    prob = {"dim": 4, "surfaces": [wl._ellipsoid([0.1, 0, 0, 0], A)], "parent": [-1], "sigma": [1.0],
            "flux": [wl.zero_flux()], "M": 2}
    with woi.Geometry(prob) as g:
        assert g.surface_area(0) == pytest.approx(core.Prepared(prob).area[0], rel=1e-10)
    # Omega_2 as printed (centre 1.4) reaches outside Omega_1
    bad = wl.ellipsoids_problem(3)
    bad["surfaces"][1]["center"][0] = 1.4
    with pytest.raises(woi.WoiError) as e:
        woi.Geometry(bad)
    assert e.value.status == 2
    # not positive definite / not symmetric / in 2D
    for M_ in ([[1.0, 0, 0], [0, -1.0, 0], [0, 0, 1.0]], [[1.0, 0.5, 0], [0, 1.0, 0], [0, 0, 1.0]]):
        with pytest.raises(woi.WoiError) as e:
            woi.woi_create_geometry(3, [wl._ellipsoid([0, 0, 0], M_)], [-1])
        assert e.value.status == 1
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(2, [wl._ellipsoid([0, 0], np.eye(2))], [-1])
    assert e.value.status == 4
    # a point charge inside the surface it sits on is not compatible (its flux integrates to -|S^{d-1}| (d-2) s)
    prob = wl.ellipsoids_problem(3)
    prob["flux"][2] = {"basis": "point_charge", "coef": [0.5, 1.6, 0.0, 0.0]}
    with pytest.raises(woi.WoiError) as e:
        woi.Geometry(prob)
    assert e.value.status == 3


def test_binding_has_every_entry_point(woi):
    """The Python binding keeps the C ABI's names: one function per declared entry point,
    and the host-only ones answer without a GPU."""
    for n in declared_entry_points():
        assert callable(getattr(woi, n, None)), n
    assert woi.woi_version()
    assert woi.woi_default_opts().M == 4
    h = woi.woi_create_geometry(3, [wl._sphere([0.0, 0.0, 0.0], 0.5)], [-1])
    try:
        assert woi.woi_surface_area(h, 0) == pytest.approx(np.pi, rel=1e-13)   # 4 pi r^2
    finally:
        woi.woi_destroy_geometry(h)
    with pytest.raises(woi.WoiError):
        woi.woi_create_geometry(3, [wl._sphere([0.0, 0.0, 0.0], -1.0)], [-1])
    assert woi.woi_last_error()


def test_mesh_inside_test_through_the_hierarchy(woi):
    """The host's inside test walks a mesh's hierarchy in the form the kernels read (both
    children's boxes in the parent's entry, a leaf child by its triangle). A sphere nested in
    a mesh is accepted only if all of its 16,384 sample points test inside: spheres within
    the polyhedron's inradius are accepted, spheres reaching beyond its circumradius are
    rejected."""
    V, F = wl.icosphere(3)                   # 1280 triangles, inradius 0.9955, circumradius 1
    for k in range(16):
        c = wl.ball_points(1, 3, 100 + k, radius=0.6)[0]
        inside = k % 2 == 0
        r = (0.985 if inside else 1.03) - float(np.linalg.norm(c))
        surfaces = [wl._mesh(V, F, [0, 0, 0]), wl._sphere(list(c), r)]
        if inside:
            woi.woi_destroy_geometry(woi.woi_create_geometry(3, surfaces, [-1, 0]))
        else:
            with pytest.raises(woi.WoiError) as e:
                woi.woi_create_geometry(3, surfaces, [-1, 0])
            assert e.value.status == 2


def test_mesh_host_geometry(woi):
    """Triangle meshes on the host side of the library: areas equal the oracle's,
    the rock workload is accepted, and open, inverted or crossing meshes are
    rejected (the crossing is found by the library's inside test)."""
    from oracle import core
    prob = wl.rocks_problem(n_rocks=3, subdiv_outer=3, subdiv_rock=2)
    prep = core.Prepared(prob)
    with woi.Geometry(prob) as g:
        for i in range(len(prob["surfaces"])):
            assert g.surface_area(i) == pytest.approx(prep.area[i], rel=1e-13)
    V, F = wl.icosphere(2)
    # an open mesh (one triangle removed)
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(3, [wl._mesh(V, F[1:], [0, 0, 0])], [-1])
    assert e.value.status == 2
    # inverted orientation
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(3, [wl._mesh(V, F[:, ::-1], [0, 0, 0])], [-1])
    assert e.value.status == 2
    # a rock crossing the outer mesh
    bad = [wl._mesh(V, F, [0, 0, 0]), wl._mesh(0.3 * V + [0.85, 0, 0], F, [0.85, 0, 0])]
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(3, bad, [-1, 0])
    assert e.value.status == 2
    # a mesh in 2D
    with pytest.raises(woi.WoiError) as e:
        woi.woi_create_geometry(2, [wl._mesh(V, F, [0, 0, 0])], [-1])
    assert e.value.status == 4
