"""Evaluation points close to an interface (GPU against the oracle).

Near a surface Phi(x, y) and grad_x Phi(x, y) are steep in the walk states y, so
the FP32 rounding of a state (the walk keeps y as an offset from its surface's
centre) and of x - c_s moves the tallies by up to about the rounding times
|grad_y Phi| |y - c| (times |D2 Phi| for the gradient).  The oracle's per-walk
error bound carries exactly these terms (pinned by the perturbation experiment of
test_oracle_error_bound.py), so the per-walk bars stay 1e-5 (FP32) and 1e-12
(FP64) of that bound at every distance.  Points at normal distance 1e-2 ... 1e-5
from a sphere (3D nested workload), a circle (2D concentric) and the star and one
of its inclusions (2D star workload), on both sides; per point 4096 replayed walks
and the estimate over the same 8192 walks (1e-2 SE), as everywhere else."""
import numpy as np
import pytest

from paper_2508_16767_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DELTAS = [1e-2, 1e-3, 1e-4, 1e-5]


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16767_gb300 import build
    build.build()
    from paper_2508_16767_gb300 import woi
    return woi


@pytest.fixture(scope="module")
def O():
    from oracle import core
    core.build()
    core.set_mutant(0)
    return core


def _cases():
    star = wl.star_inclusions_problem()
    return [("3d-nested", wl.nested_3d_problem(), [(1, -1), (1, 1), (2, -1), (2, 1), (0, -1)]),
            ("2d-concentric", wl.concentric_2d_problem(), [(1, -1), (1, 1), (0, -1)]),
            ("star-32", star, [(0, -1), (3, -1), (3, 1)])]


@pytest.mark.parametrize("case", _cases(), ids=[c[0] for c in _cases()])
def test_near_interface_walks_and_estimates(W, O, case):
    name, prob, sides = case
    M = prob["M"]
    g = W.Geometry(prob)
    ids = np.arange(4096, dtype=np.uint64)
    rows = []
    for k, (i, side) in enumerate(sides):
        x = wl.near_surface_points(prob, i, DELTAS, side, seed=31 + k)
        for dl, xp in zip(DELTAS, x):
            ov = O.walks(prob, xp, ids, seed=9, M=M, point_id=0)
            worst = {}
            for precision, bar in (("mixed", 1e-5), ("fp64", 1e-12)):
                gv = W.woi_walk_values(g, xp, ids, seed=9, point_id=0, M=M, precision=precision)
                eu = np.abs(gv["u"] - ov["u"]) / np.maximum(ov["scale"][:, 0], 1e-300)
                eg = np.max(np.abs(gv["grad"] - ov["grad"]), axis=1) / np.maximum(ov["scale"][:, 1], 1e-300)
                e = np.maximum(eu, eg)
                worst[precision] = float(e.max())
                assert e.max() <= bar, (name, i, side, dl, precision, e.max())
            rows.append((i, side, dl, worst["mixed"], worst["fp64"]))
        gr = W.woi_estimate(g, x, 8192, seed=9, M=M)
        orr = O.estimate(prob, x, 8192, seed=9, M=M)
        zu = np.abs(gr["u"] - orr["u"]) / orr["se_u"]
        zg = np.max(np.abs(gr["grad"] - orr["grad"]) / orr["se_grad"], axis=1)
        assert np.all(zu <= 1e-2) and np.all(zg <= 1e-2), (name, i, side, zu.max(), zg.max())
        for dl, a, b in zip(DELTAS, zu, zg):
            print(f"\n{name} surface {i} side {side:+d} delta {dl:.0e}: estimate |diff| / SE u {a:.2e} grad {b:.2e}")
    g.close()
    for i, side, dl, e32, e64 in rows:
        print(f"\n{name} surface {i} side {side:+d} delta {dl:.0e}: per-walk error / bound FP32 {e32:.2e} FP64 {e64:.2e}")
