"""Cross-check of the scheduled WoI estimator (Thm 4.2, the C oracle) against
the naive estimator that walks the whole Markov tree (Sec. 4.2, M = 1,
oracle/markov_tree.py): two different Monte Carlo estimators of the same
truncated series, with independent random numbers and independent code, must
agree within their combined standard error on geometries without a closed form
(an off-centre inclusion).  Planted mistakes in the schedule weights of the C
oracle break the agreement."""
import numpy as np
import pytest

from paper_2508_16767_gb300 import workloads as wl


def off_centre(d):
    c1 = np.zeros(d)
    c1[0], c1[1] = 0.3, -0.15
    if d == 2:
        flux = [wl.fourier([0.4, -0.3], [0.2, 0.5]), wl.fourier([1.0, 0.2], [-0.6, 0.1])]
    else:
        ex = tuple(1 if k == 0 else 0 for k in range(d))
        exy = tuple(1 if k < 2 else 0 for k in range(d))
        x0 = np.zeros(d)
        x0[2] = 2.5
        flux = [wl.harmonic_poly(1.0, [(1.0, ex), (0.5, exy)], d),
                {"basis": "point_charge", "coef": [0.8] + list(x0)}]
    return {"dim": d, "surfaces": [wl._sphere(np.zeros(d), 1.0), wl._sphere(c1, 0.45)], "parent": [-1, 0],
            "sigma": [1.0, 4.0], "flux": flux, "M": 1}


POINTS = {2: [[-0.5, 0.2], [0.35, -0.1], [0.0, 0.7]], 3: [[-0.5, 0.2, 0.1], [0.35, -0.1, 0.05], [0.0, 0.6, -0.3]]}


@pytest.mark.parametrize("d", [2, 3])
def test_scheduled_woi_matches_markov_tree(oracle_core, d):
    from oracle import markov_tree
    prob = off_centre(d)
    x = np.asarray(POINTS[d])
    woi = oracle_core.estimate(prob, x, 400_000, seed=11, M=1)
    for p in range(len(x)):
        m, se = markov_tree.estimate_m1(prob, x[p], 200_000, seed=100 + p)
        z = (woi["u"][p] - m) / np.hypot(woi["se_u"][p], se)
        assert abs(z) < 4.5, (d, p, woi["u"][p], m, z)


@pytest.mark.parametrize("mutant", [3, 4, 9])
def test_markov_tree_detects_schedule_mistakes(oracle_core, mutant):
    """3: no half weight at i = M; 4: no factor N; 9: H_0 drawn by |alpha|."""
    from oracle import markov_tree
    prob = off_centre(2)
    x = np.asarray(POINTS[2])
    oracle_core.set_mutant(mutant)
    try:
        woi = oracle_core.estimate(prob, x, 400_000, seed=11, M=1)
    finally:
        oracle_core.set_mutant(0)
    zs = []
    for p in range(len(x)):
        m, se = markov_tree.estimate_m1(prob, x[p], 200_000, seed=100 + p)
        zs.append(abs(woi["u"][p] - m) / np.hypot(woi["se_u"][p], se))
    assert max(zs) > 8, zs
