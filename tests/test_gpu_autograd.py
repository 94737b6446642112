"""torch.autograd through the solve: gradients of a torch loss against the oracle's VJP (GPU)."""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu


def test_autograd_gradients_match_oracle():
    import torch

    from paper_2510_16172_gb300 import build
    from paper_2510_16172_gb300.autograd import FermatSolver
    from test_gpu_parity import oracle_solve, regular

    build.build()
    oracle.build()
    sc = scenes.tiny_scene(8, n_rx=2)
    solver = FermatSolver(sc.types, 1, 2)
    tx = torch.tensor(sc.tx, dtype=torch.float64, requires_grad=True)
    rx = torch.tensor(sc.rx, dtype=torch.float64, requires_grad=True)
    verts = torch.tensor(sc.verts, dtype=torch.float64, requires_grad=True)
    X, L, status = solver(tx, rx, verts)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    ref = oracle_solve(sc, ids, order, ti, ri)
    keep = regular(ref["status"]) & (ref["minseg"] > 0.01)
    both = keep & ((status.cpu().numpy() & fpt.ST_SOLVED) > 0)
    assert both.sum() >= 0.98 * keep.sum()
    w, _ = scenes.cotangents(3, len(order), 2)
    wt = torch.as_tensor(w * both[:, None, None], dtype=torch.float32, device=X.device)
    valid = torch.as_tensor(((ref["status"] & oracle.VALID) > 0) & both, dtype=torch.float32, device=X.device)
    loss = (wt * X).sum() + (valid * L).sum()
    loss.backward()
    dL = valid.double().cpu().numpy()
    e = oracle.solve(sc, ids, order, ti, ri, dX=w * both[:, None, None], dL=dL)
    e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, e["dtheta"])
    scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), 1.0)
    np.testing.assert_allclose(tx.grad.numpy(), e_tx, atol=2e-4 * scale)
    np.testing.assert_allclose(rx.grad.numpy(), e_rx, atol=2e-4 * scale)
    np.testing.assert_allclose(verts.grad.numpy(), e_v, atol=2e-4 * scale)
