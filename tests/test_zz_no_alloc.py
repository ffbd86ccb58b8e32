"""The allocation-free estimate (woi_estimate_noalloc) against woi_estimate.

Some callers cannot allocate device memory while they run (a host framework
that owns the device heap through its own pool, real-time hosts with a memory
budget fixed at start-up, plug-ins that may only use memory handed to them).
For them the library keeps its scratch in one fixed device array.  This file
is collected last on purpose, so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process as well.
Two calls in a row must both agree with the allocating entry point (the second
call sees the first call's leftovers in the shared array)."""
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


def _check_close(a, b):
    # the tolerance of the parity tests for estimates over the same walks
    for k in ("u", "grad"):
        se = b["se_" + k].cpu().numpy()
        assert np.all(np.abs(a[k].cpu().numpy() - b[k].cpu().numpy()) <= 1e-2 * se + 1e-12), k
    for k in ("se_u", "se_grad"):
        assert np.allclose(a[k].cpu().numpy(), b[k].cpu().numpy(), rtol=1e-3), k


def test_noalloc_matches_estimate_twice(W):
    """Plain walks on spheres and circles, and the variance-reduced walk on 2D Fourier data,
    whose start draws from the beta-sign arc tables that this entry point copies into the
    fixed array; the star case puts its tables there too."""
    import torch
    star = wl.star_inclusions_problem(seed=3, n_incl=3)
    cases = [(wl.nested_3d_problem(), torch.from_numpy(wl.ball_points(200, 3, 31)).cuda(), 5000, 11, "plain"),
             (wl.concentric_2d_problem(), torch.from_numpy(wl.concentric_2d_points()).cuda(), 3000, 12, "plain"),
             (wl.concentric_2d_problem(), torch.from_numpy(wl.concentric_2d_points()).cuda(), 3000, 13, "vr"),
             (star, torch.from_numpy(wl.star_inclusions_points(star, 40, seed=5)).cuda(), 2048, 14, "vr")]
    for prob, x, n_walks, seed, variant in cases:
        g = W.Geometry(prob)
        ref = W.woi_estimate(g, x, n_walks, seed=seed, M=prob["M"], variant=variant)
        first = W.woi_estimate_noalloc(g, x, n_walks, seed=seed, M=prob["M"], variant=variant)
        second = W.woi_estimate_noalloc(g, x, n_walks, seed=seed, M=prob["M"], variant=variant)
        torch.cuda.synchronize()
        _check_close(first, ref)
        _check_close(second, ref)
        g.close()


def test_noalloc_rejects_oversized_and_host_inputs(W):
    import torch
    g = W.Geometry(wl.nested_3d_problem())
    x = torch.from_numpy(wl.ball_points(4096, 3, 12)).cuda()
    with pytest.raises(W.WoiError) as e:                      # 4096 points x 1e6 walks exceed the array
        W.woi_estimate_noalloc(g, x, 1_000_000, seed=1)
    assert e.value.status == 1
    with pytest.raises(W.WoiError) as e:                      # host points are refused
        W.woi_estimate_noalloc(g, wl.ball_points(4, 3, 1), 1024, seed=1)
    assert e.value.status == 1
    g.close()
