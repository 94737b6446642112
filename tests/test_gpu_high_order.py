"""Sequences of order 6-10 (the paper's Fig. 3 goes to n = 10) against the oracle.

Above order 5 the BFGS kernel keeps its inverse-Hessian estimate in shared
memory instead of registers, and seeded and explicit batches bucket those
sequences by order alone; enumeration, polish, validity and the implicit
backward are the same per-order kernels as below.  The tolerances are those
of the other parity tests (the backward's: twice theirs).
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes
from test_gpu_parity import check_parity, oracle_solve, regular, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


def test_enumeration_to_order_10_bit_exact(ctx):
    sc = scenes.tiny_scene(0, n_rx=2)
    sc.alphabet = np.array([0, 5, 9], dtype=np.int32)  # sum_{n=1..10} 3^n = 88,572 sequences per pair
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 10, sc.alphabet)
    ids, order, ti, ri = (t.cpu().numpy() for t in fpt.enumerate(ctx, batch))
    e = oracle.exhaustive_paths(sc, 1, 10)
    assert np.array_equal(order, e[1]) and np.array_equal(ids, e[0])
    assert np.array_equal(ti, e[2]) and np.array_equal(ri, e[3])
    sc.alphabet = np.arange(sc.n_obj, dtype=np.int32)
    sb = fpt.Batch.seeded(ctx, scene, 4242, 3000, 6, 10)
    ids, order, ti, ri = (t.cpu().numpy() for t in fpt.enumerate(ctx, sb))
    e = oracle.seeded_paths(sc, 4242, 3000, 6, 10)
    assert np.array_equal(order, e[1]) and np.array_equal(ids, e[0]) and np.array_equal(ri, e[3])


@pytest.mark.parametrize("lo,hi,seed", [(6, 6, 0), (7, 8, 1), (9, 10, 2)])
def test_seeded_high_orders_parity(ctx, lo, hi, seed):
    sc = scenes.tiny_scene(seed, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 600 + lo, 6000, lo, hi)
    out = to_np(fpt.solve(ctx, scene, batch, fpt.default_params(max_iters=64)))
    ctx.sync()
    ids, order, ti, ri = oracle.seeded_paths(sc, 600 + lo, 6000, lo, hi)
    ref = oracle_solve(sc, ids, order, ti, ri)
    assert regular(ref["status"]).sum() > 300
    check_parity(out, ref, min_solved_frac=0.98)


def test_exhaustive_batch_across_register_and_shared_memory_orders(ctx):
    """One batch holding orders 4-6: register BFGS for 4 and 5, shared-memory BFGS for 6, one output layout."""
    sc = scenes.tiny_scene(4, n_rx=2)
    sc.alphabet = np.array([0, 2, 3, 8, 10], dtype=np.int32)  # 3 planes, 2 edges
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 4, 6, sc.alphabet)
    out = to_np(fpt.solve(ctx, scene, batch))
    ctx.sync()
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 4, 6)
    ref = oracle_solve(sc, ids, order, ti, ri)
    check_parity(out, ref, min_solved_frac=0.98)
    # slots past a path's order are written as zero
    for n in (4, 5):
        sel = order == n
        assert np.all(out["T"][sel, n:] == 0) and np.all(out["X"][sel, n:] == 0)


def test_learned_start_at_high_orders(ctx):
    """An untrained network's start (slots 1-4; the later slots start at 1/2) still reaches the minimisers."""
    sc = scenes.tiny_scene(5, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    net = fpt.Mlp(ctx, 3)
    net.attach()
    batch = fpt.Batch.seeded(ctx, scene, 61, 4000, 5, 8)
    out = to_np(fpt.solve(ctx, scene, batch, fpt.default_params(init_mode=1, max_iters=64)))
    ctx.sync()
    ids, order, ti, ri = oracle.seeded_paths(sc, 61, 4000, 5, 8)
    ref = oracle_solve(sc, ids, order, ti, ri)
    check_parity(out, ref, min_solved_frac=0.97)


@pytest.mark.parametrize("lo,hi,seed", [(6, 7, 0), (8, 10, 3)])
def test_backward_high_orders(ctx, lo, hi, seed):
    """Gradients of sum w . x* + sum L* w.r.t. TX, RX and every vertex against the oracle's VJP sums."""
    import torch

    sc = scenes.tiny_scene(seed, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 700 + lo, 4000, lo, hi)
    ids, order, ti, ri = oracle.seeded_paths(sc, 700 + lo, 4000, lo, hi)
    ref = oracle_solve(sc, ids, order, ti, ri)
    keep = regular(ref["status"]) & (ref["minseg"] > 0.01)
    out = fpt.solve(ctx, scene, batch)
    ctx.sync()
    gsolved = (out["status"].cpu().numpy() & fpt.ST_SOLVED) > 0
    both = keep & gsolved
    assert both.sum() >= 0.97 * keep.sum() and both.sum() > 100
    dX, dL = scenes.cotangents(800 + lo, len(order), ids.shape[1])
    w = both.astype(np.float64)
    dX, dL = dX * w[:, None, None], dL * w
    imp = oracle.solve(sc, ids, order, ti, ri, dX=dX, dL=dL)
    e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, imp["dtheta"] * w[:, None])
    dev = out["T"].device
    g_tx, g_rx, g_v = fpt.backward(ctx, scene, batch, out["T"], None,
                                   torch.as_tensor(dX, dtype=torch.float32, device=dev),
                                   torch.as_tensor(dL, dtype=torch.float32, device=dev))
    ctx.sync()
    # twice the orders 1-3 bound: the FP32 block elimination runs through up to 10 pivot blocks
    scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), 1.0)
    np.testing.assert_allclose(g_tx.cpu().numpy(), e_tx, atol=4e-4 * scale)
    np.testing.assert_allclose(g_rx.cpu().numpy(), e_rx, atol=4e-4 * scale)
    np.testing.assert_allclose(g_v.cpu().numpy(), e_v, atol=4e-4 * scale)


def test_solve_grad_orders_1_to_10(ctx):
    """One fpt_solve_grad call over a ragged order-1..10 batch: every solved path valid per the oracle, the
    TX/RX gradients of the valid solved lengths by the envelope theorem."""
    sc = scenes.tiny_scene(6, n_rx=3)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 99, 20000, 1, 10)
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    out = fpt.alloc_outputs(ctx, batch, with_X=True)
    out, (g_tx, g_rx, g_v) = fpt.solve_grad(ctx, scene, batch, dL_status_mask=mask, out=out)
    ctx.sync()
    o = to_np(out)
    ids, order, ti, ri = oracle.seeded_paths(sc, 99, 20000, 1, 10)
    ref = oracle_solve(sc, ids, order, ti, ri)
    check_parity(o, ref, min_solved_frac=0.98)
    use = (o["status"] & mask) == mask
    assert use.sum() > 100
    e_tx = np.zeros_like(sc.tx)
    e_rx = np.zeros_like(sc.rx)
    for p in np.nonzero(use)[0]:
        n = order[p]
        first = o["X"][p, 0].astype(np.float64) - sc.tx[ti[p]]
        last = sc.rx[ri[p]] - o["X"][p, n - 1].astype(np.float64)
        e_tx[ti[p]] -= first / np.linalg.norm(first)
        e_rx[ri[p]] += last / np.linalg.norm(last)
    assert np.abs(g_tx.cpu().numpy() - e_tx).max() <= 1e-3 * max(1.0, np.abs(e_tx).max())
    assert np.abs(g_rx.cpu().numpy() - e_rx).max() <= 1e-3 * max(1.0, np.abs(e_rx).max())
