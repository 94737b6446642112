"""FP64 reference of the gradient through k unrolled solver steps -- TEST INFRASTRUCTURE ONLY.

Plain PyTorch on the CPU in float64.  The solver of Sec. III-C runs for exactly k
steps from t = 1/2 on the unified d = 2 unknowns: H_0 = I; each step takes
p = -H g, rounds of the Eq. 6 fixed point from alpha = 1 (redone from alpha = 0
when they give alpha <= 0; alpha capped at 1e3; alpha = 0 when the denominator
vanishes), t += alpha p, and the BFGS inverse update unless the curvature guard
rejects it.  The loss sum_p dX_p . X_p + dL_p L_p of the k-th iterate is then
differentiated by autograd with respect to TX, RX and the object vertices:
automatic differentiation through the iterations (Sec. IV-B), the computation the
implicit backward is compared with.

guard = "gpu": skip the update unless s^T y > 0 and (s^T y)^2 > 1e-12 |s|^2 |y|^2
(the kernels' test); guard = "c": unless s^T y > 1e-12 |s| |y| and s^T y > 0 (the
C oracle's test), which the forward pin against the C oracle uses.
"""

from __future__ import annotations

import numpy as np
import torch

QUAD = 0


def _geometry(verts, types, ids, n):
    """Per-path b [B, n, 3] and A [B, n, 3, 2] (edges: zero second column) from vertex leaves."""
    v = verts[ids[:, :n]]  # [B, n, 3, 3]
    quad = torch.as_tensor(types[ids[:, :n]] == QUAD)[..., None]
    b = v[:, :, 0]
    a1 = v[:, :, 1] - v[:, :, 0]
    a2 = torch.where(quad, v[:, :, 2] - v[:, :, 0], torch.zeros_like(a1))
    return b, torch.stack([a1, a2], dim=-1)


def _segments(b, A, tx, rx, t):
    x = b + (A @ t[..., None])[..., 0]
    pts = torch.cat([tx[:, None], x, rx[:, None]], dim=1)
    return x, pts[:, 1:] - pts[:, :-1]


def _gradient(A, z):
    u = z / z.norm(dim=-1, keepdim=True)
    d = u[:, :-1] - u[:, 1:]
    return (A.transpose(-1, -2) @ d[..., None])[..., 0].reshape(z.shape[0], -1)


def _alpha(e, qa, qc, alpha, rounds):
    for _ in range(rounds):
        w = e + alpha[:, None] * (2.0 * qa + alpha[:, None] * qc)
        r = torch.clamp(w, min=1e-30).rsqrt()
        num = (qa * r).sum(-1)
        den = (qc * r).sum(-1)
        ok = den > 1e-30
        step = torch.clamp(-num / torch.where(ok, den, torch.ones_like(den)), max=1e3)
        alpha = torch.where(ok, step, torch.zeros_like(step))
    return alpha


def unrolled_forward(b, A, tx, rx, k, fp_iters, guard="gpu"):
    """k steps of the solver; returns (t [B, n, 2], X [B, n, 3], L [B]) as differentiable tensors."""
    B, n = b.shape[0], b.shape[1]
    M = 2 * n
    t = torch.full((B, n, 2), 0.5, dtype=b.dtype)
    H = torch.eye(M, dtype=b.dtype).expand(B, M, M).clone()
    _, z = _segments(b, A, tx, rx, t)
    g = _gradient(A, z)
    for _ in range(k):
        p = -(H @ g[..., None])[..., 0]
        v = (A @ p.reshape(B, n, 2, 1))[..., 0]
        zero = torch.zeros_like(v[:, :1])
        q = torch.cat([v, zero], 1) - torch.cat([zero, v], 1)
        e = (z * z).sum(-1)
        qa = (q * z).sum(-1)
        qc = (q * q).sum(-1)
        a1 = _alpha(e, qa, qc, torch.ones(B, dtype=b.dtype), fp_iters)
        a0 = _alpha(e, qa, qc, torch.zeros(B, dtype=b.dtype), fp_iters)
        alpha = torch.where(a1 > 0, a1, a0)
        s = alpha[:, None] * p
        t = t + s.reshape(B, n, 2)
        _, z = _segments(b, A, tx, rx, t)
        gn = _gradient(A, z)
        y = gn - g
        sy = (s * y).sum(-1)
        ss = (s * s).sum(-1)
        yy = (y * y).sum(-1)
        if guard == "gpu":
            ok = (sy > 0) & (sy * sy > 1e-12 * ss * yy)
        else:
            ok = (sy > 1e-12 * torch.sqrt(ss * yy)) & (sy > 0)
        rho = 1.0 / torch.where(ok, sy, torch.ones_like(sy))
        Hy = (H @ y[..., None])[..., 0]
        yHy = (y * Hy).sum(-1)
        beta = rho * rho * yHy + rho
        wv = beta[:, None] * s - rho[:, None] * Hy
        mv = -rho[:, None] * Hy
        Hn = H + s[:, :, None] * wv[:, None, :] + mv[:, :, None] * s[:, None, :]
        H = torch.where(ok[:, None, None], Hn, H)
        g = gn
    x, z = _segments(b, A, tx, rx, t)
    return t, x, z.norm(dim=-1).sum(-1)


def unrolled_grad(scene, ids, order, tx_idx, rx_idx, k, fp_iters, dX, dL, guard="gpu"):
    """Gradients (g_tx [n_tx, 3], g_rx [n_rx, 3], g_vertices [K, 3, 3]) of sum dX . X + dL L after k steps,
    and the per-path final parameters T [M, n_max, 2].  Paths are grouped by order."""
    verts = torch.tensor(np.asarray(scene.verts, dtype=np.float64), requires_grad=True)
    tx_all = torch.tensor(np.asarray(scene.tx, dtype=np.float64), requires_grad=True)
    rx_all = torch.tensor(np.asarray(scene.rx, dtype=np.float64), requires_grad=True)
    types = np.asarray(scene.types)
    ids = np.asarray(ids)
    order = np.asarray(order)
    n_max = ids.shape[1]
    T_out = np.zeros((len(order), n_max, 2))
    loss = torch.zeros((), dtype=torch.float64)
    for n in sorted(set(order.tolist())):
        sel = np.nonzero(order == n)[0]
        if len(sel) == 0:
            continue
        b, A = _geometry(verts, types, torch.as_tensor(ids[sel]), n)
        tx = tx_all[torch.as_tensor(np.asarray(tx_idx)[sel])]
        rx = rx_all[torch.as_tensor(np.asarray(rx_idx)[sel])]
        t, x, L = unrolled_forward(b, A, tx, rx, k, fp_iters, guard)
        T_out[sel, :n] = t.detach().numpy()
        loss = loss + (torch.as_tensor(np.asarray(dX)[sel, :n]) * x).sum() + (torch.as_tensor(np.asarray(dL)[sel]) * L).sum()
    gv, gt, gr = torch.autograd.grad(loss, [verts, tx_all, rx_all], allow_unused=True)
    zero = torch.zeros
    gv = gv if gv is not None else zero(verts.shape, dtype=torch.float64)
    gt = gt if gt is not None else zero(tx_all.shape, dtype=torch.float64)
    gr = gr if gr is not None else zero(rx_all.shape, dtype=torch.float64)
    gv = gv.numpy().copy()
    gv[types != QUAD, 2] = 0.0  # an edge's third vertex slot is unused
    return gt.numpy(), gr.numpy(), gv, T_out


def unrolled_loss(scene, ids, order, tx_idx, rx_idx, k, fp_iters, dX, dL, verts=None, tx=None, rx=None,
                  guard="gpu"):
    """The loss itself (for finite differences), with optionally perturbed geometry."""
    verts = torch.tensor(np.asarray(scene.verts if verts is None else verts, dtype=np.float64))
    tx_all = torch.tensor(np.asarray(scene.tx if tx is None else tx, dtype=np.float64))
    rx_all = torch.tensor(np.asarray(scene.rx if rx is None else rx, dtype=np.float64))
    types = np.asarray(scene.types)
    ids = np.asarray(ids)
    order = np.asarray(order)
    total = 0.0
    with torch.no_grad():
        for n in sorted(set(order.tolist())):
            sel = np.nonzero(order == n)[0]
            b, A = _geometry(verts, types, torch.as_tensor(ids[sel]), n)
            tx_p = tx_all[torch.as_tensor(np.asarray(tx_idx)[sel])]
            rx_p = rx_all[torch.as_tensor(np.asarray(rx_idx)[sel])]
            _, x, L = unrolled_forward(b, A, tx_p, rx_p, k, fp_iters, guard)
            total += float((torch.as_tensor(np.asarray(dX)[sel, :n]) * x).sum() +
                           (torch.as_tensor(np.asarray(dL)[sel]) * L).sum())
    return total
