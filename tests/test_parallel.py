"""Multi-rank host logic on CPU: two gloo ranks each take a walk-range share
(their moments computed here with the oracle, as there is no GPU), the moments
are all-reduced, and the merged moments and estimate equal the single-range
run's.  The same merge through the library's walk ranges and its finalize
(woi_estimate_range, woi_finalize_moments) is a GPU test (test_gpu_multirank.py)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2508_16767_gb300 import parallel


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_walk_range_tiles():
    for world in (1, 2, 3, 8):
        for n, g in ((1000, 1), (4096, 32), (32 * 7, 32)):
            parts = [parallel.shard_walk_range(r, world, n, g, walk_begin=64) for r in range(world)]
            assert parts[0][0] == 64
            for (b0, c0), (b1, _) in zip(parts, parts[1:]):
                assert b0 + c0 == b1
            assert sum(c for _, c in parts) == n
            assert all(c % g == 0 for _, c in parts)
    with pytest.raises(ValueError):
        parallel.shard_walk_range(0, 2, 100, 32)


def _moments(est, d):
    m = np.zeros((est["sum_f"].shape[0], 2, d + 1))
    m[:, 0, :] = est["sum_f"]
    m[:, 1, :] = est["sum_gm2"]
    return m


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import core
    from paper_2508_16767_gb300 import workloads as wl
    prob = wl.concentric_2d_problem()
    x = wl.concentric_2d_points()[:6]
    b, c = parallel.shard_walk_range(rank, world, 3000, 1)
    est = core.estimate(prob, x, c, seed=9, M=4, walk_begin=b)
    merged = parallel.allreduce_moments(_moments(est, 2))
    np.save(os.path.join(out_dir, f"merged{rank}.npy"), merged)
    dist.destroy_process_group()


def test_two_rank_gloo_merge(tmp_path):
    from oracle import core
    from paper_2508_16767_gb300 import workloads as wl
    core.build()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    m0 = np.load(tmp_path / "merged0.npy")
    m1 = np.load(tmp_path / "merged1.npy")
    assert np.array_equal(m0, m1)
    prob = wl.concentric_2d_problem()
    x = wl.concentric_2d_points()[:6]
    full = core.estimate(prob, x, 3000, seed=9, M=4)
    assert np.allclose(m0, _moments(full, 2), rtol=1e-12, atol=1e-13)
    # per-walk schedules: the group means are the walks' values, so sum_gm = sum_f
    f = core.finalize(m0[:, 0, :], m0[:, 0, :], m0[:, 1, :], 3000, 3000)
    assert np.allclose(f["u"], full["u"], rtol=1e-12, atol=1e-13)
    assert np.allclose(f["se_u"], full["se_u"], rtol=1e-9)
