"""FP64 reference of the warm-start network -- TEST INFRASTRUCTURE ONLY.

Plain numpy, following the network's definition (include/fpt.h): BF16 inputs
and weights, accumulation (here FP64), bias + GELU in its tanh form, activations
rounded to BF16 between layers, and for the gradient the same rounding points
as the definition fixes (dY and dZ enter the products as BF16, bias gradients
use the unrounded dZ).  With round_bf16=False everything stays FP64, which the
finite-difference pins use.
"""

from __future__ import annotations

import numpy as np
N_IN, N_H, N_OUT = 64, 256, 16
SIZES = [("W1", (256, 64)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)), ("b3", (256,)),
         ("W4", (16, 256)), ("b4", (16,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(flat):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16(x):
    """Round to bfloat16 (round to nearest even on the float32 bit pattern), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


K0 = np.sqrt(2.0 / np.pi)
K1 = 0.044715


def gelu(z):
    """GELU, tanh form (Hendrycks and Gimpel): z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(K0 * (z + K1 * z ** 3)))


def gelu_grad(z):
    th = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * K0 * (1.0 + 3.0 * K1 * z * z)


def features(scene, ids, order, tx_idx, rx_idx, scale):
    """The 64 features of each path and the per-slot Gram matrices (definition in include/fpt.h), FP64.

    Per interaction: the parameters tau of the orthogonal projections of TX and
    RX onto the object's affine hull (least squares in the object's basis), their
    distances to it, |a1| and the distance-weighted mean of the two projections.
    """
    M = len(order)
    F = np.zeros((M, N_IN))
    G = np.zeros((M, 4, 3))
    for p in range(M):
        tx, rx = scene.tx[tx_idx[p]], scene.rx[rx_idx[p]]
        o = 0.5 * (tx + rx)
        F[p, 0:3] = (tx - o) / scale
        F[p, 3:6] = (rx - o) / scale
        for s in range(min(int(order[p]), 4)):
            k = ids[p, s]
            v0, v1, v3 = scene.verts[k]
            edge = scene.types[k] == 1
            a1 = v1 - v0
            a2 = np.zeros(3) if edge else v3 - v0
            A = a1[:, None] if edge else np.stack([a1, a2], axis=1)
            tau, dist = [], []
            for pt in (tx, rx):
                c = np.linalg.lstsq(A, pt - v0, rcond=None)[0]
                t2 = np.zeros(2)
                t2[:len(c)] = c
                tau.append(t2)
                dist.append(np.linalg.norm(pt - v0 - A @ c) / scale)
            base = 6 + 11 * s
            F[p, base] = 1.0
            F[p, base + 1] = 1.0 if edge else 0.0
            F[p, base + 2:base + 4] = tau[0]
            F[p, base + 4:base + 6] = tau[1]
            F[p, base + 6:base + 8] = dist
            F[p, base + 8] = np.linalg.norm(a1) / scale
            ds = dist[0] + dist[1]
            F[p, base + 9:base + 11] = ((dist[1] * tau[0] + dist[0] * tau[1]) / ds) if ds > 0 else 0.5 * (tau[0] + tau[1])
            G[p, s] = [a1 @ a1 / scale ** 2, a1 @ a2 / scale ** 2, a2 @ a2 / scale ** 2]
    return F, G


def forward(params, X, round_bf16=True):
    P = unpack(params)
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    acts = {"X": r(X)}
    h = acts["X"]
    for l in (1, 2, 3):
        z = h @ r(P[f"W{l}"]).T + P[f"b{l}"]
        acts[f"Z{l}"] = z
        h = r(gelu(z))
        acts[f"H{l}"] = h
    acts["Y"] = h @ r(P["W4"]).T + P["b4"]
    return acts


def loss_and_dY(G, Y, T):
    """Loss of the definition, (1/B) sum_b sum_s dy_s^T G_s dy_s, and its gradient with respect to Y (FP64)."""
    B = len(Y)
    d = (Y[:, :8] - T).reshape(B, 4, 2)
    m = np.stack([G[:, :, 0] * d[:, :, 0] + G[:, :, 1] * d[:, :, 1], G[:, :, 1] * d[:, :, 0] + G[:, :, 2] * d[:, :, 1]],
                 axis=2)
    loss = np.sum(d * m) / B
    dY = np.zeros_like(Y)
    dY[:, :8] = 2.0 * m.reshape(B, 8) / B
    return loss, dY


def loss_grad(params, X, T, G, round_bf16=True):
    """Loss and gradient with respect to the flat parameters."""
    P = unpack(params)
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    A = forward(params, X, round_bf16)
    Xr = A["X"]
    loss, dY = loss_and_dY(G, A["Y"], T)
    grads = {}
    dYr = r(dY)
    grads["W4"] = dYr.T @ A["H3"]
    grads["b4"] = dY.sum(axis=0)
    dZ = (dYr @ r(P["W4"])) * gelu_grad(A["Z3"])
    for l in (3, 2, 1):
        grads[f"b{l}"] = dZ.sum(axis=0)
        dZr = r(dZ)
        inp = A[f"H{l - 1}"] if l > 1 else Xr
        grads[f"W{l}"] = dZr.T @ inp
        if l > 1:
            dZ = (dZr @ r(P[f"W{l}"])) * gelu_grad(A[f"Z{l - 1}"])
    return loss, pack(grads)
