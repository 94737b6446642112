"""torch.autograd.Function around the solve and its implicit-differentiation backward.

    solver = FermatSolver(types, order_lo=1, order_hi=2)
    X, L, status = solver(tx, rx, verts)       # tx [n_tx,3], rx [n_rx,3], verts [K,3,3]
    loss = (L * ((status & fpt.ST_VALID) > 0)).sum()
    loss.backward()                             # gradients for tx, rx and verts

Forward runs fpt_solve on every exhaustive candidate sequence; backward runs
fpt_backward with the incoming cotangents of X and L (Sec. III-D: solve
H u = -v per path, then u^T d(grad_T L)/d(theta) plus the explicit terms).
Paths that are repeats, degenerate, non-finite or invalid carry no gradient.

The geometry stays on the GPU: the solver keeps one scene whose records are
rebuilt from the CUDA tensors by the library's kernels (fpt_scene_upload_device
on the first call, then fpt_scene_update_vertices and fpt_set_endpoints_device),
so no call copies TX, RX or vertices to the host or waits for the device.  A
backward whose forward is not the most recent one first restores that
forward's geometry (saved on the device).  Marshalling only: both directions
run in libfpt.so.
"""

from __future__ import annotations

import numpy as np
import torch

from . import fpt


class _FermatPathsFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, tx, rx, verts, solver):
        geo = tuple(t.detach().to(device=solver.device, dtype=torch.float32).contiguous() for t in (tx, rx, verts))
        scene, batch, version = solver._load(*geo)
        out = fpt.solve(solver.ctx, scene, batch, solver.params)
        fctx.solver, fctx.version = solver, version
        fctx.in_meta = [(t.dtype, t.device) for t in (tx, rx, verts)]
        fctx.save_for_backward(out["T"], out["status"], *geo)
        fctx.mark_non_differentiable(out["status"])
        return out["X"], out["L"], out["status"]

    @staticmethod
    def backward(fctx, dX, dL, _dstatus):
        T, status, tx, rx, verts = fctx.saved_tensors
        solver = fctx.solver
        if solver.version != fctx.version:  # a later forward replaced the geometry: restore this one's
            solver._load(tx, rx, verts)
        dX = dX.contiguous().float() if dX is not None else None
        dL = dL.contiguous().float() if dL is not None else None
        g_tx, g_rx, g_v = fpt.backward(solver.ctx, solver.scene, solver.batch, T, status, dX, dL)
        outs = []
        for g, (dt, dev) in zip((g_tx, g_rx, g_v), fctx.in_meta):
            outs.append(g.to(device=dev, dtype=dt))
        return outs[0], outs[1], outs[2], None


class FermatSolver:
    """Differentiable batched Fermat path solve over all sequences of order lo..hi.

    centre: the point (3 floats, metres) the library recentres the geometry on for FP32
    precision; None = the origin.
    """

    def __init__(self, types, order_lo=1, order_hi=2, alphabet=None, params=None, device=0, centre=None):
        self.ctx = fpt.Context(device)
        self.device = torch.device("cuda", device)
        self.types = np.ascontiguousarray(types, dtype=np.uint8)
        self.order_lo, self.order_hi = order_lo, order_hi
        self.alphabet = alphabet
        self.params = params if params is not None else fpt.default_params()
        self.centre = None if centre is None else np.asarray(centre, dtype=np.float64).reshape(3)
        self.scene = None
        self.batch = None
        self.version = 0

    def _load(self, tx, rx, verts):
        """Put this geometry (CUDA float32 tensors) into the solver's scene; returns (scene, batch, version)."""
        if self.scene is None:
            self.scene = fpt.Scene(self.ctx, self.types, verts, centre=self.centre)
        else:
            self.scene.update_vertices(verts)
        counts = (self.scene.n_tx, self.scene.n_rx)
        self.scene.set_endpoints(tx, rx)
        if self.batch is None or counts != (self.scene.n_tx, self.scene.n_rx):
            if self.batch is not None:
                self.batch.close()
            self.batch = fpt.Batch.exhaustive(self.ctx, self.scene, self.order_lo, self.order_hi, self.alphabet)
        self.version += 1
        return self.scene, self.batch, self.version

    def __call__(self, tx, rx, verts):
        return _FermatPathsFn.apply(tx, rx, verts, self)
