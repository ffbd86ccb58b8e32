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
