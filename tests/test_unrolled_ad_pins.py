"""Pins of the FP64 unrolled-AD reference (oracle/unrolled_ad.py).

Its forward is the C oracle's implementation of the paper's solver run for a
fixed step count; its gradient is the derivative of that forward (central
differences); and for a converged run it meets the implicit-function gradient
of the solution (the oracle's VJP).
"""

import numpy as np
import pytest

import oracle
from oracle import unrolled_ad
from paper_2510_16172_gb300 import scenes


def _paths(seed, lo=1, hi=3):
    sc = scenes.tiny_scene(seed)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, lo, hi)
    # skip immediate repeats (never solved)
    keep = np.array([all(ids[p, i] != ids[p, i + 1] for i in range(order[p] - 1)) for p in range(len(order))])
    return sc, ids[keep], order[keep], ti[keep], ri[keep]


@pytest.mark.parametrize("fp", [1, 4])
def test_forward_is_the_c_oracles_solver(oracle_lib, fp):
    sc, ids, order, ti, ri = _paths(5, 1, 2)
    k = 10
    dX = np.zeros((len(order), ids.shape[1], 3))
    dL = np.zeros(len(order))
    *_, T = unrolled_ad.unrolled_grad(sc, ids, order, ti, ri, k, fp, dX, dL, guard="c")
    ref = oracle.solve(sc, ids, order, ti, ri, solver=oracle.BFGS, max_iters=k, fp_iters=fp, tol_step=0.0)
    ok = (ref["status"] & oracle.DEGENERATE) == 0
    assert ok.sum() > 0.9 * len(order)
    for p in np.nonzero(ok)[0]:
        n = order[p]
        np.testing.assert_allclose(T[p, :n], ref["T"][p, :n], rtol=0, atol=1e-9)


def test_gradient_is_the_derivative_of_the_forward(oracle_lib):
    sc, ids, order, ti, ri = _paths(6, 1, 3)
    rng = np.random.default_rng(1)
    sel = rng.choice(len(order), 60, replace=False)
    ids, order, ti, ri = ids[sel], order[sel], ti[sel], ri[sel]
    dX, dL = scenes.cotangents(3, len(order), ids.shape[1])
    k, fp = 8, 2
    g_tx, g_rx, g_v, _ = unrolled_ad.unrolled_grad(sc, ids, order, ti, ri, k, fp, dX, dL)
    h = 1e-6
    checks = [("v", 0, 0, 0), ("v", 3, 1, 2), ("v", 9, 0, 1), ("v", 10, 1, 0), ("tx", 0, 0, 2), ("rx", 0, 0, 1)]
    for kind, o, vtx, c in checks:
        def loss(sign):
            verts, tx, rx = sc.verts.copy(), sc.tx.copy(), sc.rx.copy()
            if kind == "v":
                verts[o, vtx, c] += sign * h
            elif kind == "tx":
                tx[o, c] += sign * h
            else:
                rx[o, c] += sign * h
            return unrolled_ad.unrolled_loss(sc, ids, order, ti, ri, k, fp, dX, dL, verts=verts, tx=tx, rx=rx)

        fd = (loss(1) - loss(-1)) / (2 * h)
        got = g_v[o, vtx, c] if kind == "v" else (g_tx[o, c] if kind == "tx" else g_rx[o, c])
        assert abs(fd - got) <= 1e-5 * max(1.0, abs(fd)), (kind, o, vtx, c, fd, got)


def test_converged_run_meets_the_implicit_gradient(oracle_lib):
    """Differentiating enough iterations reproduces the implicit-function gradient of the minimiser."""
    sc, ids, order, ti, ri = _paths(7, 1, 2)
    ref = oracle.solve(sc, ids, order, ti, ri)
    X = ref["X"]
    minseg = np.array([np.linalg.norm(np.diff(np.vstack([sc.tx[ti[p]], X[p, :order[p]], sc.rx[ri[p]]]), axis=0),
                                      axis=1).min() for p in range(len(order))])
    keep = ((ref["status"] & oracle.CONVERGED) > 0) & ((ref["status"] & oracle.DEGENERATE) == 0) & (minseg > 0.05)
    ids, order, ti, ri = ids[keep], order[keep], ti[keep], ri[keep]
    dX, dL = scenes.cotangents(4, len(order), ids.shape[1])
    g_tx, g_rx, g_v, _ = unrolled_ad.unrolled_grad(sc, ids, order, ti, ri, 120, 1, dX, dL)
    imp = oracle.solve(sc, ids, order, ti, ri, dX=dX, dL=dL)
    e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, imp["dtheta"])
    scale = max(np.abs(e_v).max(), 1.0)
    np.testing.assert_allclose(g_v, e_v, atol=1e-6 * scale)
    np.testing.assert_allclose(g_tx, e_tx, atol=1e-6 * scale)
    np.testing.assert_allclose(g_rx, e_rx, atol=1e-6 * scale)
