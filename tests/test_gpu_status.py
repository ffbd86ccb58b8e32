"""Status reporting of conditions found on the device.

A line or ray that crosses one mesh more than 32 times overflows the kernel's
bounded crossing list: the extra crossings are dropped (never written past the
list) and counted, and the call that ran those walks must report
WOI_E_GEOMETRY -- synchronous calls in their own status, asynchronous calls
(device points and outputs) through woi_check_status, and batches in theirs.
The counter is per call: a later call on a well-behaved geometry reports OK."""
import numpy as np
import pytest

from paper_2508_16767_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2508_16767_gb300 import build
    build.build()
    from paper_2508_16767_gb300 import woi
    return woi


def test_mesh_crossing_overflow_is_reported_on_every_path(W):
    import torch
    prob = wl.bellows_problem()
    x = np.array([[0.0, 0.0, 0.05], [0.1, -0.1, 0.0]])
    g = W.Geometry(prob)
    with pytest.raises(W.WoiError) as e:                      # synchronous: host outputs
        W.woi_estimate(g, x, 4096, seed=1)
    assert e.value.status == 2
    xd = torch.from_numpy(x).cuda()
    W.woi_estimate(g, xd, 4096, seed=1)                       # asynchronous: returns before the kernels end
    with pytest.raises(W.WoiError) as e:
        W.woi_check_status(g)
    assert e.value.status == 2
    W.woi_check_status(g)                                     # read once
    with pytest.raises(W.WoiError) as e:                      # batch
        W.woi_estimate_batch([(g, xd, 4096)], seed=1)
    assert e.value.status == 2
    with pytest.raises(W.WoiError) as e:                      # pathwise replay
        W.woi_walk_values(g, x[0], np.arange(4096, dtype=np.uint64), seed=1, M=prob["M"])
    assert e.value.status == 2
    g.close()
    # a mesh geometry whose lines stay within the list: every path reports OK
    rocks = wl.rocks_problem(n_rocks=3, subdiv_outer=3, subdiv_rock=2, M=4)
    g = W.Geometry(rocks)
    xr = torch.from_numpy(wl.mesh_points(rocks, 4, seed=61)).cuda()
    W.woi_estimate(g, xr, 4096, seed=1)
    W.woi_check_status(g)
    g.close()
