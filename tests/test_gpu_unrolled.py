"""fpt_backward_unrolled: reverse-mode differentiation through a fixed number of solver steps.

Its forward must be the unified solver run for exactly k steps (bit for bit),
and its gradient that of the FP64 autograd reference through the same steps
(oracle/unrolled_ad.py): the per-object sums after a few steps, and each
path's own gradient, in distribution, through more steps.
"""

import numpy as np
import pytest

import oracle
from oracle import unrolled_ad
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


def _no_repeat(ids, order):
    return np.array([all(ids[p, i] != ids[p, i + 1] for i in range(order[p] - 1)) for p in range(len(order))])


def _dev(x):
    import torch

    return torch.as_tensor(x, dtype=torch.float32, device="cuda:0")


@pytest.mark.parametrize("fp,lo,hi", [(1, 1, 3), (4, 1, 3), (1, 6, 10)])
def test_forward_is_the_solver_at_a_fixed_step_count(ctx, fp, lo, hi):
    """The taped forward takes the unified kernel's steps: the same iterates to the bit."""
    sc = scenes.tiny_scene(1, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, lo, hi) if hi <= 3 else fpt.Batch.seeded(ctx, scene, 5, 3000, lo, hi)
    k = 12
    *_, T, st = fpt.backward_unrolled(ctx, scene, batch, k, fp, want_T=True)
    p = fpt.default_params(max_iters=k, fixed_iters=1, fp_iters=fp, polish=0, specialize=0, kink_stop=1e-30)
    out = fpt.solve(ctx, scene, batch, p)
    ctx.sync()
    s_st = out["status"].cpu().numpy()
    run = (s_st & (fpt.ST_REPEAT | fpt.ST_INVALID_INPUT | fpt.ST_NONFINITE)) == 0
    assert run.sum() > 0.5 * len(s_st)
    assert np.array_equal(T.cpu().numpy()[run], out["T"].cpu().numpy()[run])
    skip = (s_st & fpt.ST_REPEAT) > 0
    assert np.array_equal(st.cpu().numpy()[skip] & fpt.ST_REPEAT, s_st[skip] & fpt.ST_REPEAT)


@pytest.mark.parametrize("fp", [1, 4])
@pytest.mark.parametrize("seed", range(4))
def test_summed_gradient_matches_the_fp64_autograd_reference(ctx, seed, fp):
    """Gradients w.r.t. TX, RX and every vertex of sum dX . X_k + dL L_k over every sequence of
    order 1-3 (shared objects: the per-object sums), after k = 2 steps, where FP32 and FP64 runs of
    the same steps still agree to about 1e-5 of the largest gradient."""
    sc = scenes.tiny_scene(seed, n_rx=2)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 3)
    k = 2
    use = _no_repeat(ids, order)
    dX, dL = scenes.cotangents(300 + seed, len(order), ids.shape[1])
    dX, dL = dX * use[:, None, None], dL * use
    g_tx, g_rx, g_v, _, st = fpt.backward_unrolled(ctx, scene, batch, k, fp, _dev(dX), _dev(dL))
    e_tx, e_rx, e_v, _ = unrolled_ad.unrolled_grad(sc, ids[use], order[use], ti[use], ri[use], k, fp, dX[use],
                                                   dL[use])
    ctx.sync()
    assert not (st.cpu().numpy() & fpt.ST_NONFINITE).any()
    scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), np.abs(e_rx).max(), 1.0)
    for got, ref in ((g_tx, e_tx), (g_rx, e_rx), (g_v, e_v)):
        err = np.abs(got.cpu().numpy() - ref).max() / scale
        assert err < 2e-4, err


def _private_scene(sc, ids, order, ti, ri):
    """Every path gets its own copies of its objects and endpoints, so that the scene-level
    gradients are the paths' own gradients."""
    types, verts, tx, rx = [], [], [], []
    nids = np.full_like(ids, -1)
    for p in range(len(order)):
        for i in range(order[p]):
            nids[p, i] = len(types)
            types.append(sc.types[ids[p, i]])
            verts.append(sc.verts[ids[p, i]])
        tx.append(sc.tx[ti[p]])
        rx.append(sc.rx[ri[p]])
    idx = np.arange(len(order))
    return scenes.Scene(np.array(types), np.array(verts), np.array(tx), np.array(rx)), nids, idx, idx


# (k, Eq. 6 rounds, paths, orders, fraction within 1e-3, fraction within 1e-2, median bound).  Measured on the
# GB300 with these seeds (the gradients are deterministic: every path has its own objects): 100 % within 1e-3
# at k = 4 and at orders 6-10; at k = 16, 87.3 % / 96.0 % (one round) and 84.0 % / 93.6 % (four rounds) within
# 1e-3 / 1e-2; medians 9e-7 to 1.4e-5.  A CPU FP32 run of the reference reaches 86 % and 80 % within 1e-3 at
# k = 16, so the bounds sit just below what any FP32 evaluation of these iterations gets.
@pytest.mark.parametrize("k,fp,n_paths,lo,hi,min_frac,min_frac2,max_median", [
    (4, 1, 300, 1, 3, 0.99, 1.0, 5e-6), (16, 1, 300, 1, 3, 0.82, 0.93, 5e-5), (16, 4, 700, 1, 3, 0.78, 0.90, 6e-5),
    (4, 1, 200, 6, 8, 0.99, 1.0, 8e-6), (8, 1, 200, 6, 8, 0.98, 1.0, 5e-5), (4, 4, 200, 9, 10, 0.99, 1.0, 5e-6)])
def test_per_path_gradients_against_the_fp64_autograd_reference(ctx, k, fp, n_paths, lo, hi, min_frac, min_frac2,
                                                                  max_median):
    """Each path's gradient w.r.t. its own geometry against the FP64 reference through the same k steps.

    Differentiating BFGS through FP32 iterations is ill-conditioned once steps near the rounding
    level enter the inverse-Hessian updates (rho = 1 / s.y): a CPU FP32 run of the same autograd
    reference departs from the FP64 one by more than 1e-3 of the gradient on 14-20 % of these
    paths at k = 16 while most agree to 1e-5.  The test asks for that distribution: fractions of
    the paths within 1e-3 and within 1e-2 (relative to the path's largest gradient component, at
    least 1) and a small median.  700 paths put the scene's accumulators in global memory, 300 in shared memory; orders
    6-10 keep the inverse Hessian and its adjoint in shared memory (a CPU FP32 run of the reference
    is within 1e-3 on all of those paths).
    """
    import torch

    base = scenes.tiny_scene(5, n_rx=2)
    if hi <= 3:
        ids, order, ti, ri = oracle.exhaustive_paths(base, lo, hi)
    else:
        ids, order, ti, ri = oracle.seeded_paths(base, 77, 2000, lo, hi)
    ok = np.nonzero(_no_repeat(ids, order))[0]
    sel = np.sort(np.random.default_rng(k + fp).choice(ok, n_paths, replace=False))
    sc, nids, ti2, ri2 = _private_scene(base, ids[sel], order[sel], ti[sel], ri[sel])
    order = order[sel]
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.explicit(ctx, scene, torch.as_tensor(nids, dtype=torch.int32, device="cuda"),
                               torch.as_tensor(order, dtype=torch.uint8, device="cuda"),
                               torch.as_tensor(ti2, dtype=torch.int32, device="cuda"),
                               torch.as_tensor(ri2, dtype=torch.int32, device="cuda"))
    dX, dL = scenes.cotangents(40 + k, len(order), nids.shape[1])
    g_tx, g_rx, g_v, _, st = fpt.backward_unrolled(ctx, scene, batch, k, fp, _dev(dX), _dev(dL))
    e_tx, e_rx, e_v, _ = unrolled_ad.unrolled_grad(sc, nids, order, ti2, ri2, k, fp, dX, dL)
    ctx.sync()
    g_tx, g_rx, g_v = g_tx.cpu().numpy(), g_rx.cpu().numpy(), g_v.cpu().numpy()
    rel = np.empty(len(order))
    for p in range(len(order)):
        o = nids[p, :order[p]]
        got = np.concatenate([g_v[o].ravel(), g_tx[p], g_rx[p]])
        ref = np.concatenate([e_v[o].ravel(), e_tx[p], e_rx[p]])
        rel[p] = np.abs(got - ref).max() / max(np.abs(ref).max(), 1.0)
    rel[~np.isfinite(rel)] = np.inf
    assert (rel < 1e-3).mean() >= min_frac, (np.sort(rel)[::-1][:10], (rel < 1e-3).mean())
    assert (rel < 1e-2).mean() >= min_frac2, (np.sort(rel)[::-1][:10], (rel < 1e-2).mean())
    assert np.median(rel) < max_median, np.median(rel)


def test_zero_steps_and_argument_errors(ctx):
    """k = 0: the gradient of the loss at the start t = 1/2; bad step and round counts are argument errors."""
    import torch

    sc = scenes.tiny_scene(0)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 2)
    # zero steps: the gradient of the loss at the start t = 1/2
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    keep = _no_repeat(ids, order)
    dX, dL = scenes.cotangents(5, len(order), ids.shape[1])
    dX, dL = dX * keep[:, None, None], dL * keep
    g_tx, g_rx, g_v, T, _ = fpt.backward_unrolled(ctx, scene, batch, 0, 1, _dev(dX),
                                                  _dev(dL), want_T=True)
    e_tx, e_rx, e_v, _ = unrolled_ad.unrolled_grad(sc, ids[keep], order[keep], ti[keep], ri[keep], 0, 1, dX[keep],
                                                   dL[keep])
    ctx.sync()
    scale = max(np.abs(e_v).max(), 1.0)
    assert np.abs(g_v.cpu().numpy() - e_v).max() < 1e-5 * scale
    assert np.abs(g_tx.cpu().numpy() - e_tx).max() < 1e-5 * scale
    Tn = T.cpu().numpy()
    for p in np.nonzero(keep)[0]:
        assert np.all(Tn[p, :order[p], 0] == 0.5)
    for bad in ((-1, 1), (4097, 1), (4, 0), (4, 65)):
        with pytest.raises(fpt.FptError):
            fpt.backward_unrolled(ctx, scene, batch, *bad)
    with pytest.raises((fpt.FptError, TypeError, ValueError)):
        fpt.backward_unrolled(ctx, scene, batch, 4, 1, dX=torch.zeros(3))
