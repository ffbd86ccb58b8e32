"""Walk-range sharding through the library on two ranks (GPU).

Two processes (gloo ranks on the host) each run their share of the walks of
every point with woi_estimate_range on the GPU; the raw moments are all-reduced
on the host and finalized by the library (woi_finalize_moments).  The merged
estimate must equal a single call over all walks up to the order of the FP64
sums, and the oracle's estimate over the same walks within the parity bar.  The
ranks' kernels never wait on each other: the only exchange is the host
all-reduce between steps."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    from paper_2508_16767_gb300 import workloads as wl
    return wl.nested_3d_problem(), wl.ball_points(40, 3, 77)


N_WALKS = 6144


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2508_16767_gb300 import parallel, woi
    prob, x = _problem()
    b, c = parallel.shard_walk_range(rank, world, N_WALKS, 32)
    g = woi.Geometry(prob)
    mom = woi.woi_estimate_range(g, torch.from_numpy(x).cuda(), b, c, seed=6, M=prob["M"], sched_group=32)
    torch.cuda.synchronize()
    merged = parallel.allreduce_moments(mom.cpu())           # host all-reduce between steps
    f = parallel.finalize(merged.cuda(), N_WALKS, 32)        # the library's finalize kernel
    torch.cuda.synchronize()
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), **{k: v.cpu().numpy() for k, v in f.items()},
             moments=merged.numpy())
    g.close()
    dist.destroy_process_group()


def test_two_rank_ranges_merge_through_the_library(tmp_path):
    import torch
    import torch.multiprocessing as mp
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16767_gb300 import build
    build.build()
    from oracle import core
    core.build()
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r0, r1 = np.load(tmp_path / "r0.npz"), np.load(tmp_path / "r1.npz")
    for k in ("u", "grad", "se_u", "se_grad", "moments"):
        assert np.array_equal(r0[k], r1[k]), k
    from paper_2508_16767_gb300 import woi
    prob, x = _problem()
    g = woi.Geometry(prob)
    single = woi.woi_estimate(g, x, N_WALKS, seed=6, M=prob["M"], sched_group=32)
    g.close()
    for k in ("u", "grad", "se_u", "se_grad"):
        assert np.allclose(r0[k], single[k], rtol=1e-12, atol=1e-12 * np.abs(single[k]).max()), k
    orr = core.estimate(prob, x, N_WALKS, seed=6, M=prob["M"], sched_group=32)
    assert np.all(np.abs(r0["u"] - orr["u"]) <= 1e-2 * orr["se_u"])
    assert np.all(np.abs(r0["grad"] - orr["grad"]) <= 1e-2 * orr["se_grad"])
    assert np.allclose(r0["se_u"], orr["se_u"], rtol=1e-3)


def test_finalize_moments_host_and_device():
    """woi_finalize_moments with host and device arrays against the single call."""
    import torch
    from paper_2508_16767_gb300 import build
    build.build()
    from paper_2508_16767_gb300 import woi
    prob, x = _problem()
    g = woi.Geometry(prob)
    mom = woi.woi_estimate_range(g, x, 0, 4096, seed=2, M=prob["M"])
    single = woi.woi_estimate(g, x, 4096, seed=2, M=prob["M"])
    g.close()
    host = woi.woi_finalize_moments(mom, 4096)
    dev = woi.woi_finalize_moments(torch.from_numpy(mom).cuda(), 4096)
    torch.cuda.synchronize()
    for k in ("u", "grad", "se_u", "se_grad"):
        assert np.array_equal(host[k], dev[k].cpu().numpy()), k
        assert np.allclose(host[k], single[k], rtol=1e-13, atol=0), k
    with pytest.raises(woi.WoiError) as e:
        woi.woi_finalize_moments(mom, 4016, sched_group=32)   # not a multiple of the group
    assert e.value.status == 1
