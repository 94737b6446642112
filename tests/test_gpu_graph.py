"""fpt_solve_grad captured in a CUDA graph and replayed (the step of a serving loop).

Every launch of the call -- the pattern kernels on their side streams included -- goes into the
capture; counts such as the polish's second-pass list live on the device, so nothing reads back
to the host.  The replay must give the outputs of a direct call bit for bit.
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


@pytest.mark.parametrize("workload", ["canyon", "tiny-seeded"])
def test_solve_grad_graph_replay_matches_direct_call(ctx, workload):
    import torch

    if workload == "canyon":
        sc = scenes.urban_canyon(0, rx_grid=8)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    else:
        sc = scenes.tiny_scene(2, n_rx=2)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.seeded(ctx, scene, 17, 20000, 1, 7)
    p = fpt.default_params(max_iters=32)
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    direct, (dtx, drx, dv) = fpt.solve_grad(ctx, scene, batch, p, dL_status_mask=mask)
    ctx.sync()
    ref = {k: v.clone() for k, v in direct.items() if v is not None}
    ref_g = (dtx.clone(), drx.clone(), dv.clone())
    out = fpt.alloc_outputs(ctx, batch)
    grads = (torch.empty_like(dtx), torch.empty_like(drx), torch.empty_like(dv))
    fpt.solve_grad(ctx, scene, batch, p, dL_status_mask=mask, out=out, grads=grads)  # warm-up: workspaces
    ctx.sync()
    g = torch.cuda.CUDAGraph()
    old = ctx.stream
    with torch.cuda.graph(g):
        ctx.set_stream(torch.cuda.current_stream())
        fpt.solve_grad(ctx, scene, batch, p, dL_status_mask=mask, out=out, grads=grads)
    ctx.set_stream(old)
    for k in out:
        if out[k] is not None:
            out[k].zero_()
    for t in grads:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for k, v in ref.items():
        assert torch.equal(out[k], v), k
    for a, b in zip(grads, ref_g):
        # sums of per-path terms in FP64 atomics: the order of additions may differ between runs
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-5 * float(b.abs().max()))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out["T"], ref["T"])
