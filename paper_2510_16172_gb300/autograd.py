"""torch.autograd.Function around the solve and its implicit-differentiation backward.

    solver = FermatSolver(types, order_lo=1, order_hi=2)
    X, L, status = solver(tx, rx, verts)       # tx [n_tx,3], rx [n_rx,3], verts [K,3,3]
    loss = (L * ((status & fpt.ST_VALID) > 0)).sum()
    loss.backward()                             # gradients for tx, rx and verts

Forward runs fpt_solve on every exhaustive candidate sequence; backward runs
fpt_backward with the incoming cotangents of X and L (Sec. III-D: solve
H u = -v per path, then u^T d(grad_T L)/d(theta) plus the explicit terms).
Paths that are repeats, degenerate, non-finite or invalid carry no gradient.
Marshalling only: both directions run in libfpt.so.
"""

from __future__ import annotations

import numpy as np
import torch

from . import fpt


class _FermatPathsFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, tx, rx, verts, solver):
        scene = fpt.Scene(solver.ctx, solver.types, verts.detach().cpu().double().numpy(),
                          tx.detach().cpu().double().numpy(), rx.detach().cpu().double().numpy())
        batch = fpt.Batch.exhaustive(solver.ctx, scene, solver.order_lo, solver.order_hi, solver.alphabet)
        out = fpt.solve(solver.ctx, scene, batch, solver.params)
        fctx.scene, fctx.batch, fctx.solver = scene, batch, solver
        fctx.in_meta = [(t.dtype, t.device) for t in (tx, rx, verts)]
        fctx.save_for_backward(out["T"], out["status"])
        fctx.mark_non_differentiable(out["status"])
        return out["X"], out["L"], out["status"]

    @staticmethod
    def backward(fctx, dX, dL, _dstatus):
        T, status = fctx.saved_tensors
        dX = dX.contiguous().float() if dX is not None else None
        dL = dL.contiguous().float() if dL is not None else None
        g_tx, g_rx, g_v = fpt.backward(fctx.solver.ctx, fctx.scene, fctx.batch, T, status, dX, dL)
        outs = []
        for g, (dt, dev) in zip((g_tx, g_rx, g_v), fctx.in_meta):
            outs.append(g.to(device=dev, dtype=dt))
        return outs[0], outs[1], outs[2], None


class FermatSolver:
    """Differentiable batched Fermat path solve over all sequences of order lo..hi."""

    def __init__(self, types, order_lo=1, order_hi=2, alphabet=None, params=None, device=0):
        self.ctx = fpt.Context(device)
        self.types = np.ascontiguousarray(types, dtype=np.uint8)
        self.order_lo, self.order_hi = order_lo, order_hi
        self.alphabet = alphabet
        self.params = params if params is not None else fpt.default_params()

    def __call__(self, tx, rx, verts):
        return _FermatPathsFn.apply(tx, rx, verts, self)
