"""Writes replay_small.json: per-walk values of the FP64 oracle on tiny cases
(only oracle/ and the input generator are called).  Run from the repository
root:  python tests/golden/make_replay.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import core  # noqa: E402
from paper_2508_16767_gb300 import workloads as wl  # noqa: E402


def cases():
    yield "2d-concentric", wl.concentric_2d_problem(), wl.concentric_2d_points()[[3, 40]], "plain", 4
    yield "3d-nested", wl.nested_3d_problem(), wl.ball_points(2, 3, 12), "plain", 6
    yield "star-3", wl.star_inclusions_problem(seed=3, n_incl=3), np.array([[0.1, 0.2], [-0.5, 0.3]]), "plain", 3
    yield "star-3-vr", wl.star_inclusions_problem(seed=3, n_incl=3), np.array([[0.6, -0.4]]), "vr", 3
    yield "3d-linear-vr", wl.linear_3d_problem(), wl.ball_points(1, 3, 5, radius=0.9), "vr", 4
    yield "3d-zonal-vr", wl.zonal_3d_problem(), wl.ball_points(1, 3, 6, radius=0.9), "vr", 4
    yield "4d-nested", wl.nested_nd_problem(4), wl.ball_points(1, 4, 7), "plain", 4
    yield "5d-nested-vr", wl.nested_nd_problem(5), wl.ball_points(1, 5, 8, radius=0.9), "vr", 4
    yield "6d-nested", wl.nested_6d_problem(), wl.ball_points(1, 6, 9), "plain", 4
    ell4 = wl.ellipsoids_problem(4)
    yield "ellipsoids-4d", ell4, wl.ellipsoid_points(ell4, 1, seed=10), "plain", 3


def main():
    out = {"_source": "oracle/core.py walks(), seed 0, walks 0..31", "cases": []}
    for name, prob, x, variant, M in cases():
        for p, xp in enumerate(x):
            r = core.walks(prob, xp, np.arange(32), seed=0, M=M, variant=variant, point_id=p)
            out["cases"].append({"name": name, "variant": variant, "M": M, "point_id": p, "x": xp.tolist(),
                                 "u": r["u"].tolist(), "grad": r["grad"].tolist(), "H": r["H"].tolist()})
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "replay_small.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
