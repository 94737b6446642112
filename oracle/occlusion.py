"""Obstruction of solved paths by the scene's planar objects -- TEST INFRASTRUCTURE ONLY.

Sec. I: a candidate ray is discarded when it is obstructed, as well as when an
interaction point falls outside its object.  Plain numpy in float64, written
from that definition:

  * Segment j (j = 0..n) of a path of order n runs from x_j to x_{j+1}, with
    x_0 = TX and x_{n+1} = RX.
  * The objects at its two ends (slot j-1 and slot j of the sequence) never
    block it; an edge (a line) blocks nothing.
  * A planar object (the closed parallelogram b + u a1 + v a2, 0 <= u, v <= 1)
    blocks the segment when the segment crosses its plane properly -- the two
    ends are on opposite sides, each more than `tol` metres from the plane --
    and the crossing point lies in the parallelogram.

blocked_segments() returns, per path, a bit mask (bit j set: segment j is
blocked).  Its `grow` argument widens every parallelogram by that many metres
along its plane on all sides (negative: shrinks it): the decision is monotone
in `grow` and in `tol`, so decided() can mark the paths whose masks do not
change when the points move by a small amount -- the cases that a different
rounding, or a solution 1e-4 m away, may not decide the other way.
"""

from __future__ import annotations

import numpy as np

QUAD = 0


def _quads(scene):
    v = np.asarray(scene.verts, dtype=np.float64)
    types = np.asarray(scene.types)
    idx = np.nonzero(types == QUAD)[0]
    b = v[idx, 0]
    a1 = v[idx, 1] - v[idx, 0]
    a2 = v[idx, 2] - v[idx, 0]
    nrm = np.cross(a1, a2)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return idx, b, a1, a2, nrm


def _in_plane_coords(h, b, a1, a2):
    """(u, v) with h - b = u a1 + v a2 (h in the plane), by the 2 x 2 normal equations."""
    r = h - b
    g11 = (a1 * a1).sum(-1)
    g12 = (a1 * a2).sum(-1)
    g22 = (a2 * a2).sum(-1)
    r1 = (r * a1).sum(-1)
    r2 = (r * a2).sum(-1)
    det = g11 * g22 - g12 * g12
    return (g22 * r1 - g12 * r2) / det, (g11 * r2 - g12 * r1) / det


def blocked_segments(scene, ids, order, tx_idx, rx_idx, X, tol=1e-4, grow=0.0):
    """Bit masks [M] (uint16) of blocked segments."""
    ids = np.asarray(ids)
    order = np.asarray(order)
    X = np.asarray(X, dtype=np.float64)
    qidx, b, a1, a2, nrm = _quads(scene)
    # in-plane distance between the sides u = 0 and u = 1 is area / |a2|, between v = 0 and v = 1 area / |a1|
    area = np.linalg.norm(np.cross(a1, a2), axis=1)
    gu = grow / (area / np.linalg.norm(a2, axis=1))
    gv = grow / (area / np.linalg.norm(a1, axis=1))
    masks = np.zeros(len(order), dtype=np.uint16)
    for p in range(len(order)):
        n = int(order[p])
        pts = np.vstack([scene.tx[tx_idx[p]], X[p, :n], scene.rx[rx_idx[p]]])
        for j in range(n + 1):
            P, Q = pts[j], pts[j + 1]
            own = set()
            if j >= 1:
                own.add(int(ids[p, j - 1]))
            if j < n:
                own.add(int(ids[p, j]))
            keep = np.array([int(o) not in own for o in qidx])
            if not keep.any():
                continue
            dP = ((P - b[keep]) * nrm[keep]).sum(-1)
            dQ = ((Q - b[keep]) * nrm[keep]).sum(-1)
            cross = ((dP > tol) & (dQ < -tol)) | ((dP < -tol) & (dQ > tol))
            s = dP / np.where(cross, dP - dQ, 1.0)
            h = P + s[:, None] * (Q - P)
            u, v = _in_plane_coords(h, b[keep], a1[keep], a2[keep])
            inside = (u >= -gu[keep]) & (u <= 1 + gu[keep]) & (v >= -gv[keep]) & (v <= 1 + gv[keep])
            if np.any(cross & inside):
                masks[p] |= np.uint16(1 << j)
    return masks


def decided(scene, ids, order, tx_idx, rx_idx, X, tol=1e-4, plane=0.5e-4, side=1e-3):
    """Paths whose masks stay the same when the plane tolerance moves by +-plane metres and the
    parallelograms grow or shrink by `side` metres."""
    most = blocked_segments(scene, ids, order, tx_idx, rx_idx, X, tol - plane, side)
    least = blocked_segments(scene, ids, order, tx_idx, rx_idx, X, tol + plane, -side)
    return most == least
