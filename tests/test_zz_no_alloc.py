"""fpt_backward_noalloc: the backward for callers that cannot allocate device memory (GPU).

Some callers cannot call cudaMalloc: their GPU memory belongs to another
allocator, or their loop must not allocate.  This entry point keeps its
scratch in a fixed array inside the library.  Its results must equal the
regular fpt_backward's, call after call, since every call reuses (and must
clear) the same array.  Collected last, so a run that stops at the first
failure has already run every other test.
"""

import numpy as np
import pytest

from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2510_16172_gb300 import build

    build.build()
    return fpt.Context(0)


def compare(a, b):
    scale = max(1.0, max(float(x.abs().max()) for x in b))
    for x, y in zip(a, b):
        np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), atol=2e-4 * scale)


@pytest.mark.parametrize("workload", ["tiny", "canyon"])
def test_noalloc_backward_matches_backward_twice(ctx, workload):
    import torch

    if workload == "tiny":
        sc = scenes.tiny_scene(4, n_rx=3)
        lo, hi = 1, 3
    else:
        sc = scenes.urban_canyon(0, rx_grid=4)  # 16 RX x 32^3 = 524,288 order-3 paths
        lo = hi = 3
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, lo, hi, sc.alphabet)
    out = fpt.solve(ctx, scene, batch)
    dX, dL = scenes.cotangents(9, batch.n_paths, batch.n_max)
    dX = torch.as_tensor(dX, dtype=torch.float32, device="cuda")
    dL = torch.as_tensor(dL, dtype=torch.float32, device="cuda")
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    # the caller owns the outputs, as a caller that cannot allocate would
    got = (torch.empty((scene.n_tx, 3), dtype=torch.float32, device="cuda"),
           torch.empty((scene.n_rx, 3), dtype=torch.float32, device="cuda"),
           torch.empty((scene.n_obj, 3, 3), dtype=torch.float32, device="cuda"))
    for k in range(2):  # two calls in a row: the fixed array keeps the previous call's contents
        ref = fpt.backward(ctx, scene, batch, out["T"], out["status"], dX, dL)
        fpt.backward_noalloc(ctx, scene, batch, out["T"], out["status"], dX, dL, out=got)
        ctx.sync()
        compare(got, ref)
        ref = fpt.backward(ctx, scene, batch, out["T"], out["status"], None, None, dL_status_mask=mask)
        fpt.backward_noalloc(ctx, scene, batch, out["T"], out["status"], None, None, dL_status_mask=mask, out=got)
        ctx.sync()
        compare(got, ref)
    # further calls take no device memory: the free memory the driver reports stays the same
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(3):
        fpt.backward_noalloc(ctx, scene, batch, out["T"], out["status"], dX, dL, out=got)
        fpt.backward_noalloc(ctx, scene, batch, out["T"], out["status"], None, None, dL_status_mask=mask, out=got)
    ctx.sync()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_backward_rejects_sizes_beyond_its_limit(ctx):
    sc = scenes.urban_canyon(0, rx_grid=6)  # 36 RX x 32^3 = 1,179,648 paths of order 3 > 2^20
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    import torch

    T = torch.zeros((batch.n_paths, 3, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(fpt.FptError, match="limit"):
        fpt.backward_noalloc(ctx, scene, batch, T)
