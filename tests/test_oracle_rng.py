"""Pins of the oracle's random-number layer (CPU)."""
import ctypes
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_core):
    for ctr, key, out in _kat():
        assert list(oracle_core.philox4x32_10(ctr, key)) == out


def _curand_host():
    for path in ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"]:
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator(oracle_core):
    """cuRAND's host Philox4_32_10 generator emits philox((0, 0, j, 0), seed) for
    tuple j; running it (a library, on the CPU) pins the round function and the
    key schedule for keys with both words set."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    for seed in [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF]:
        gen = ctypes.c_void_p()
        if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:
            pytest.skip("cuRAND host generator unavailable")
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 2048
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        lib.curandDestroyGenerator(gen)
        out = out.reshape(-1, 4)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for j in list(range(8)) + list(range(100, 2048, 97)):
            assert list(oracle_core.philox4x32_10([0, 0, j, 0], key)) == list(out[j])


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_directions_isotropic(oracle_core, d):
    """Unit vectors with mean 0 and second moment I/d (isotropy, Sec. 4.2.3)."""
    n = 20000
    z = oracle_core.directions(d, n, seed=11)
    assert np.allclose(np.linalg.norm(z, axis=1), 1.0, atol=1e-12)
    assert np.abs(z.mean(axis=0)).max() < 5.0 / np.sqrt(n)
    C = z.T @ z / n
    assert np.abs(C - np.eye(d) / d).max() < 6.0 * np.sqrt(2.0 / (d * d * n)) + 1e-3


def _schedule_from_word(thresh, n, i, w):
    """Thm 4.2's schedule from a 32-bit word: H_0 uniform over the n surfaces, H_i (i >= 1)
    the first surface whose threshold exceeds the word."""
    if i == 0:
        return (w * n) >> 32
    for k in range(n):
        if w < int(thresh[k]):
            return k
    return n - 1


@pytest.mark.parametrize("name,sched_group", [("2d-circles", 1), ("2d-circles", 32), ("2d-star", 1), ("3d", 1),
                                              ("3d", 32)])
def test_schedule_words_follow_the_protocol(oracle_core, name, sched_group):
    """The oracle's schedules H_i against the random-number protocol written out here from its
    definition: key = (seed_lo ^ point, seed_hi ^ instance); the schedule word of step i of a
    walk is word 0 of the call (walk, i, chain 0 | sub 0), except on 2D instances whose surfaces
    are all circles, where steps 2j and 2j + 1 share the call (walk, j, 0) and take its words 0
    and 2; with W_g = 32 every walk of a group takes the group leader's (walk 32 g) word."""
    from paper_2508_16767_gb300 import workloads as wl
    if name == "2d-circles":
        prob, x = wl.concentric_2d_problem(), np.array([0.3, -0.2])
    elif name == "2d-star":
        prob, x = wl.star_inclusions_problem(seed=3, n_incl=3), np.array([0.1, 0.2])
    else:
        prob, x = wl.nested_3d_problem(), np.array([0.1, 0.2, -0.3])
    paired = prob["dim"] == 2 and all(s["kind"] == "sphere" for s in prob["surfaces"])
    M, seed, point_id, instance = prob["M"], (5 << 32) | 77, 3, 2
    walks = np.concatenate([np.arange(64), 2 ** 33 + np.arange(32)]).astype(np.uint64)
    tr = oracle_core.walks(prob, x, walks, seed=seed, M=M, sched_group=sched_group, point_id=point_id,
                           instance=instance)
    alpha, _ = oracle_core.alpha_beta_scale(np.asarray(prob["sigma"]), prob["parent"])
    thresh, _ = oracle_core.schedule_thresholds(alpha)
    n = len(prob["surfaces"])
    key = [(seed ^ point_id) & 0xFFFFFFFF, ((seed >> 32) ^ instance) & 0xFFFFFFFF]
    for r, w in enumerate(walks):
        lead = int(w) // sched_group * sched_group
        for i in range(M + 1):
            step, word = (i >> 1, 2 * (i & 1)) if paired else (i, 0)
            words = oracle_core.philox4x32_10([lead & 0xFFFFFFFF, lead >> 32, step, 0], key)
            assert tr["H"][r, i] == _schedule_from_word(thresh, n, i, int(words[word])), (name, int(w), i)
