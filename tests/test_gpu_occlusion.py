"""fpt_occlusion against the obstruction oracle (oracle/occlusion.py).

The GPU tests its own solved points; the oracle tests the oracle's.  Bits are
compared exactly on the paths both solve, where the oracle's decision does not
change when the plane tolerance moves by 5e-5 m or the parallelograms grow or
shrink by 1 mm (the two sets of points are at most 1e-4 m apart).
"""

import numpy as np
import pytest

import oracle
from oracle import occlusion
from paper_2510_16172_gb300 import fpt, scenes
from test_gpu_parity import oracle_solve, regular

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


def _compare(ctx, sc, scene, batch, ids, order, ti, ri, sample=None):
    out = fpt.solve(ctx, scene, batch)
    bits = fpt.occlusion(ctx, scene, batch, out["T"])
    ctx.sync()
    st = out["status"].cpu().numpy()
    bits = bits.cpu().numpy().astype(np.uint16)
    if sample is not None:
        st, bits = st[sample], bits[sample]
    ref = oracle_solve(sc, ids, order, ti, ri)
    ob = occlusion.blocked_segments(sc, ids, order, ti, ri, ref["X"])
    use = regular(ref["status"]) & ((st & fpt.ST_SOLVED) > 0) & occlusion.decided(sc, ids, order, ti, ri, ref["X"])
    assert use.sum() > 100
    bad = np.nonzero(bits[use] != ob[use])[0]
    assert len(bad) == 0, (len(bad), bits[use][bad[:5]], ob[use][bad[:5]])
    return use, ob


@pytest.mark.parametrize("seed", range(3))
def test_tiny_scenes_orders_1_to_3(ctx, seed):
    sc = scenes.tiny_scene(seed, n_quads=12, n_edges=4, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 3)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
    use, ob = _compare(ctx, sc, scene, batch, ids, order, ti, ri)
    assert (ob[use] != 0).mean() > 0.05  # a real share of the compared paths is obstructed


def test_seeded_high_orders(ctx):
    sc = scenes.tiny_scene(7, n_quads=12, n_edges=4, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 808, 3000, 4, 8)
    ids, order, ti, ri = oracle.seeded_paths(sc, 808, 3000, 4, 8)
    use, ob = _compare(ctx, sc, scene, batch, ids, order, ti, ri)
    assert (ob[use] != 0).mean() > 0.05


def test_urban_canyon_sampled(ctx):
    sc = scenes.urban_canyon(0, rx_grid=8)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    g = np.sort(np.random.default_rng(3).choice(batch.n_paths, 4000, replace=False))
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 3, 3, g)
    _compare(ctx, sc, scene, batch, ids, order, ti, ri, sample=g)


def test_status_mask_and_arguments(ctx):
    import torch

    sc = scenes.tiny_scene(1, n_quads=12, n_edges=4)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 2)
    out = fpt.solve(ctx, scene, batch)
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    all_bits = fpt.occlusion(ctx, scene, batch, out["T"])
    some = fpt.occlusion(ctx, scene, batch, out["T"], out["status"], mask)
    ctx.sync()
    sel = ((out["status"] & mask) == mask).cpu().numpy()
    a, m = all_bits.cpu().numpy(), some.cpu().numpy()
    assert np.array_equal(m[sel], a[sel]) and not m[~sel].any()
    rep = (out["status"].cpu().numpy() & fpt.ST_REPEAT) > 0
    assert not a[rep].any()
    with pytest.raises(fpt.FptError):
        fpt.occlusion(ctx, scene, batch, out["T"], None, mask)
    with pytest.raises(fpt.FptError):
        fpt.occlusion(ctx, scene, batch, out["T"], tol=-1.0)
    with pytest.raises(fpt.FptError):
        fpt.occlusion(ctx, scene, batch, out["T"], out=torch.zeros(3, dtype=torch.int16, device="cuda"))
