"""The backward's per-warp sums against the oracle for every way a warp's lanes can share targets (GPU).

The adjoint kernel adds each path's gradient terms into per-object, per-TX and per-RX accumulators.
Before adding, the lanes of a warp that share a target are summed onto one lane: by a butterfly when
every lane has the same target, by a segmented scan when the groups are contiguous runs of lanes, and
otherwise by pulling one group member per round.  An exhaustive order-1 batch over an alphabet of k
facades of the city scene, with 64 receivers, fixes which case each sum meets: consecutive paths run
through the alphabet for one receiver, so a warp's object targets form k scattered groups of 32 / k
lanes (one group for k = 1, 32 different targets for k = 32) and its receiver targets form runs of k
lanes.  The summed TX, RX and vertex gradients are compared with the oracle's implicit VJP (Sec. III-D,
Eq. 9-13) summed over the same paths, both with point cotangents (every path in index order) and with
length cotangents alone (the adjoint runs over the list of paths that carry one).
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    return fpt.Context(0)


def regular(st):
    return ((st & oracle.CONVERGED) > 0) & ((st & (oracle.DEGENERATE | oracle.REPEAT | oracle.NONFINITE)) == 0)


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16, 32])
def test_warp_sums_by_target_grouping(ctx, k):
    import torch

    sc = scenes.city(0, n_rx=64)
    sc.alphabet = np.nonzero(sc.types == scenes.QUAD)[0][:k].astype(np.int32)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 1, sc.alphabet)
    out = fpt.solve(ctx, scene, batch)
    ctx.sync()
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 1)
    assert len(order) == 64 * k
    ref0 = oracle.solve(sc, ids, order, ti, ri)
    pts = np.stack([sc.tx[ti], ref0["X"][:, 0], sc.rx[ri]], axis=1)
    minseg = np.linalg.norm(np.diff(pts, axis=1), axis=2).min(axis=1)
    gsolved = (out["status"].cpu().numpy() & fpt.ST_SOLVED) > 0
    both = regular(ref0["status"]) & (minseg > 0.01) & gsolved
    assert both.mean() > 0.95  # order-1 paths off facade planes: nearly all regular, so the groups stay intact
    dX, dL = scenes.cotangents(11 + k, len(order), 1)
    w = both.astype(np.float64)
    dX, dL = dX * w[:, None, None], dL * w
    dev = out["T"].device
    for with_points in (True, False):
        dXk = dX if with_points else None
        ref = oracle.solve(sc, ids, order, ti, ri, dX=dXk, dL=dL)
        e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, ref["dtheta"])
        g_tx, g_rx, g_v = fpt.backward(
            ctx, scene, batch, out["T"], out["status"],
            torch.as_tensor(dXk, dtype=torch.float32, device=dev) if with_points else None,
            torch.as_tensor(dL, dtype=torch.float32, device=dev))
        ctx.sync()
        scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), np.abs(e_rx).max(), 1.0)
        for got, want, what in ((g_tx, e_tx, "TX"), (g_rx, e_rx, "RX"), (g_v, e_v, "vertices")):
            np.testing.assert_allclose(got.cpu().numpy(), want, atol=2e-4 * scale,
                                       err_msg=f"{what}, k = {k}, point cotangents: {with_points}")
