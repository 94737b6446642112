"""fpt_solve_grad: solve and implicit backward in one call (adjoint after the solve, or fused into the polish).

Its outputs must be those of fpt_solve, and its gradients those of the
oracle's VJP (same tolerance as fpt_backward) and of fpt_solve followed by
fpt_backward.
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu

MASK = fpt.ST_VALID | fpt.ST_SOLVED


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


def _regular(st):
    return ((st & oracle.CONVERGED) > 0) & ((st & (oracle.DEGENERATE | oracle.REPEAT | oracle.NONFINITE)) == 0)


def _min_segments(sc, order, ti, ri, X):
    out = np.full(len(order), np.inf)
    for p in range(len(order)):
        n = order[p]
        pts = np.vstack([sc.tx[ti[p]], X[p, :n], sc.rx[ri[p]]])
        out[p] = np.linalg.norm(np.diff(pts, axis=0), axis=1).min()
    return out


@pytest.mark.parametrize("fuse", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_solve_grad_matches_oracle_vjp(ctx, seed, fuse):
    """Gradients of sum_i w_i . x_i* + sum L* w.r.t. TX, RX and every vertex against the oracle VJP."""
    import torch

    sc = scenes.tiny_scene(seed, n_rx=2)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    ref = oracle.solve(sc, ids, order, ti, ri)
    keep = _regular(ref["status"]) & (_min_segments(sc, order, ti, ri, ref["X"]) > 0.01)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 2)
    first = fpt.solve(ctx, scene, batch)
    gsolved = (first["status"].cpu().numpy() & fpt.ST_SOLVED) > 0
    both = keep & gsolved
    assert both.sum() >= 0.98 * keep.sum()
    dX, dL = scenes.cotangents(200 + seed, len(order), 2)
    w = both.astype(np.float64)
    dX = dX * w[:, None, None]
    dL = np.where((ref["status"] & oracle.VALID) > 0, 1.0, 0.3 * dL) * w
    ref = oracle.solve(sc, ids, order, ti, ri, dX=dX, dL=dL)
    e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, ref["dtheta"])
    dev = first["T"].device
    out, (g_tx, g_rx, g_v) = fpt.solve_grad(ctx, scene, batch, fpt.default_params(fuse_adjoint=fuse),
                                            dX=torch.as_tensor(dX, dtype=torch.float32, device=dev),
                                            dL=torch.as_tensor(dL, dtype=torch.float32, device=dev))
    ctx.sync()
    assert np.array_equal(out["status"].cpu().numpy(), first["status"].cpu().numpy())
    scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), 1.0)
    np.testing.assert_allclose(g_tx.cpu().numpy(), e_tx, atol=2e-4 * scale)
    np.testing.assert_allclose(g_rx.cpu().numpy(), e_rx, atol=2e-4 * scale)
    np.testing.assert_allclose(g_v.cpu().numpy(), e_v, atol=2e-4 * scale)


@pytest.mark.parametrize("fuse", [0, 1])
@pytest.mark.parametrize("case", ["canyon", "city"])
def test_solve_grad_equals_solve_then_backward(ctx, case, fuse):
    """Same outputs as fpt_solve, same sums as fpt_backward (valid-length mask plus seeded point cotangents)."""
    import torch

    if case == "canyon":
        sc = scenes.urban_canyon(0, rx_grid=4)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    else:
        sc = scenes.city(3, n_rx=4)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.seeded(ctx, scene, 11, 20000, 1, 5)
    a = fpt.solve(ctx, scene, batch)
    # point cotangents on paths whose segments are all >= 1 cm: near a kink the adjoint amplifies rounding
    # differences by 1/|z|, which would let a few paths dominate the comparison of the sums
    dev = a["T"].device
    Xa = a["X"].double()
    _, order, txi, rxi = fpt.enumerate(ctx, batch)
    ends_tx = torch.as_tensor(sc.tx, device=dev)[txi.long()]
    ends_rx = torch.as_tensor(sc.rx, device=dev)[rxi.long()]
    order = order.long()
    pts = torch.cat([ends_tx[:, None], Xa, ends_rx[:, None]], dim=1)
    idx = torch.arange(batch.n_max + 2, device=dev)[None, :]
    inner = ((idx >= 1) & (idx <= order[:, None]))[:, :, None]
    pts = torch.where(inner, pts, ends_rx[:, None].expand_as(pts))
    pts[:, 0] = ends_tx
    seg = (pts[:, 1:] - pts[:, :-1]).norm(dim=2)
    last = torch.arange(batch.n_max + 1, device=dev)[None, :] <= order[:, None]
    far = torch.where(last, seg, torch.full_like(seg, 1e9)).min(dim=1).values >= 0.01
    dX = torch.as_tensor(scenes.cotangents(5, batch.n_paths, batch.n_max)[0], dtype=torch.float32, device=dev)
    dX = (dX * 0.1 * far[:, None, None]).contiguous()
    ref = fpt.backward(ctx, scene, batch, a["T"], a["status"], dX, None, dL_status_mask=MASK)
    b, got = fpt.solve_grad(ctx, scene, batch, fpt.default_params(fuse_adjoint=fuse), dX=dX, dL_status_mask=MASK)
    ctx.sync()
    assert np.array_equal(a["iters"].cpu().numpy(), b["iters"].cpu().numpy())
    # the two polish instantiations may round a Newton step differently, which can flip a borderline flag
    st_a, st_b = a["status"].cpu().numpy(), b["status"].cpu().numpy()
    assert np.count_nonzero(st_a != st_b) <= 1e-4 * len(st_a)
    # the two polish instantiations may round a Newton step differently: on solved paths (a well-defined
    # stationary point) the results agree to the parity bounds; unsolved ones need not agree
    solved = ((st_a & st_b) & fpt.ST_SOLVED) > 0
    np.testing.assert_allclose(b["X"].cpu().numpy()[solved], a["X"].cpu().numpy()[solved], rtol=0, atol=1e-4)
    np.testing.assert_allclose(b["L"].cpu().numpy()[solved], a["L"].cpu().numpy()[solved], rtol=1e-6, atol=0)
    for r, g, name in zip(ref, got, ("g_tx", "g_rx", "g_vertices")):
        r, g = r.cpu().numpy(), g.cpu().numpy()
        scale = max(np.abs(r).max(), 1.0)
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-3 * scale, err_msg=name)


def test_solve_grad_argument_errors(ctx):
    sc = scenes.tiny_scene(1)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 2)
    with pytest.raises(fpt.FptError):
        fpt.solve_grad(ctx, scene, batch, fpt.default_params(polish=0), dL_status_mask=MASK)
    with pytest.raises(fpt.FptError):
        fpt.solve_grad(ctx, scene, batch, fpt.default_params(polish_fp64=1), dL_status_mask=MASK)
    with pytest.raises(fpt.FptError):
        fpt.solve_grad(ctx, scene, batch, fpt.default_params(polish=0, fuse_adjoint=1), dL_status_mask=MASK)
    ctx.sync()
