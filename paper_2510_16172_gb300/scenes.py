"""Seeded synthetic scene generators (numpy only).

These build the inputs of the batched Fermat path solve: planar reflectors
(parallelograms given by three corners) and straight diffraction edges (two
end points), plus transmitter (TX) and receiver (RX) positions.  The paper
evaluates on random scenes it does not specify (Sec. IV); these generators are
the stand-in, one per workload:

* ``tiny_scene``   -- a 10 m box with 8 random rectangles (sides 1-4 m,
  uniform orientation) and 4 random edges (length 1-3 m), one TX and one RX
  uniform in the box.  All R/D sequences of order 1-2 over its 12 objects.
* ``urban_canyon`` -- 32 vertical axis-aligned facade rectangles (5-30 m) on a
  200 x 200 m grid plus their 4 boundary edges each, TX at (100, 100, 10) m,
  a 32 x 32 RX grid at 1.5 m, and a 32-object alphabet of 16 facades and 16
  of their edges (32^3 order-3 sequences per TX/RX pair).
* ``city``         -- a 500 x 500 x 60 m block of facades and edges used for
  ragged, seed-sampled batches.

This module holds no part of the method's arithmetic: it only draws geometry.
Both the CUDA path and the CPU oracle consume what it returns.

Object encoding (shared by every consumer):
  type 0 = QUAD (planar reflector): verts[k] = (v0, v1, v3), a parallelogram
           with corners v0, v1, v1 + v3 - v0, v3.
  type 1 = EDGE (straight wedge):   verts[k] = (e0, e1, unused zeros).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

QUAD = 0
EDGE = 1


@dataclass
class Scene:
    """A scene: objects, endpoints and the alphabet sequences are drawn from."""

    types: np.ndarray  # uint8 [K]
    verts: np.ndarray  # float64 [K, 3, 3]
    tx: np.ndarray  # float64 [n_tx, 3]
    rx: np.ndarray  # float64 [n_rx, 3]
    alphabet: np.ndarray = field(default=None)  # int32 [n_alpha] object ids

    def __post_init__(self):
        self.types = np.ascontiguousarray(self.types, dtype=np.uint8)
        self.verts = np.ascontiguousarray(self.verts, dtype=np.float64)
        self.tx = np.ascontiguousarray(np.atleast_2d(self.tx), dtype=np.float64)
        self.rx = np.ascontiguousarray(np.atleast_2d(self.rx), dtype=np.float64)
        if self.alphabet is None:
            self.alphabet = np.arange(len(self.types), dtype=np.int32)
        self.alphabet = np.ascontiguousarray(self.alphabet, dtype=np.int32)

    @property
    def n_obj(self) -> int:
        return int(len(self.types))


def _unit(rng: np.random.Generator) -> np.ndarray:
    """Uniform direction on the unit sphere (normalised Gaussian)."""
    while True:
        v = rng.standard_normal(3)
        n = np.linalg.norm(v)
        if n > 1e-6:
            return v / n


def _perp_basis(n: np.ndarray, phi: float) -> tuple[np.ndarray, np.ndarray]:
    """Orthonormal in-plane pair (u, v) of the plane with normal n, rotated by phi."""
    helper = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u0 = np.cross(n, helper)
    u0 /= np.linalg.norm(u0)
    v0 = np.cross(n, u0)
    u = np.cos(phi) * u0 + np.sin(phi) * v0
    v = -np.sin(phi) * u0 + np.cos(phi) * v0
    return u, v


def random_rectangle(rng, side_lo, side_hi, centre_lo, centre_hi) -> np.ndarray:
    """Rectangle with uniform normal, uniform in-plane rotation and sides U[lo, hi]."""
    n = _unit(rng)
    u, v = _perp_basis(n, rng.uniform(0.0, 2.0 * np.pi))
    w, h = rng.uniform(side_lo, side_hi, size=2)
    c = rng.uniform(centre_lo, centre_hi, size=3)
    v0 = c - 0.5 * w * u - 0.5 * h * v
    return np.stack([v0, v0 + w * u, v0 + h * v])


def random_edge(rng, len_lo, len_hi, centre_lo, centre_hi) -> np.ndarray:
    """Segment with uniform direction, length U[lo, hi] and uniform midpoint."""
    d = _unit(rng)
    ln = rng.uniform(len_lo, len_hi)
    m = rng.uniform(centre_lo, centre_hi, size=3)
    return np.stack([m - 0.5 * ln * d, m + 0.5 * ln * d, np.zeros(3)])


def tiny_scene(seed: int, n_quads: int = 8, n_edges: int = 4, n_tx: int = 1, n_rx: int = 1) -> Scene:
    """10 m box: rectangles (side 1-4 m, centre U[1,9]^3), edges (1-3 m), TX/RX U[0,10]^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    verts = [random_rectangle(rng, 1.0, 4.0, 1.0, 9.0) for _ in range(n_quads)]
    verts += [random_edge(rng, 1.0, 3.0, 1.0, 9.0) for _ in range(n_edges)]
    types = [QUAD] * n_quads + [EDGE] * n_edges
    tx = rng.uniform(0.0, 10.0, size=(n_tx, 3))
    rx = rng.uniform(0.0, 10.0, size=(n_rx, 3))
    return Scene(np.array(types), np.array(verts), tx, rx)


def _facade(rng, extent: float, grid: float, w_lo: float, w_hi: float, h_lo: float, h_hi: float):
    """Vertical axis-aligned rectangle standing on z = 0, its plane on a street grid."""
    axis = int(rng.integers(0, 2))  # 0: plane x = const (normal +-x), 1: plane y = const
    w = rng.uniform(w_lo, w_hi)
    h = rng.uniform(h_lo, h_hi)
    n_lines = int(round(extent / grid))
    plane = grid * float(rng.integers(1, n_lines))  # on a grid line, off the border
    along = rng.uniform(0.5 * w, extent - 0.5 * w)
    if axis == 0:
        v0 = np.array([plane, along - 0.5 * w, 0.0])
        a1 = np.array([0.0, w, 0.0])
    else:
        v0 = np.array([along - 0.5 * w, plane, 0.0])
        a1 = np.array([w, 0.0, 0.0])
    a2 = np.array([0.0, 0.0, h])
    return np.stack([v0, v0 + a1, v0 + a2])


def _facade_edges(q: np.ndarray) -> list[np.ndarray]:
    """The 4 boundary edges of parallelogram (v0, v1, v3): bottom, top, left, right."""
    v0, v1, v3 = q
    v2 = v1 + v3 - v0
    z = np.zeros(3)
    return [np.stack([v0, v1, z]), np.stack([v3, v2, z]), np.stack([v0, v3, z]), np.stack([v1, v2, z])]


def urban_canyon(seed: int = 0, n_facades: int = 32, rx_grid: int = 32, n_alpha_quads: int = 16,
                 n_alpha_edges: int = 16, extent: float = 200.0) -> Scene:
    """Urban canyon: facades (5-30 m) on a 200 x 200 m grid, their edges, a TX and an RX grid.

    Objects: n_facades rectangles followed by their 4 edges each.  The alphabet
    mixes a seeded choice of n_alpha_quads facades (reflections) and
    n_alpha_edges of the vertical/top edges (diffractions).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    quads = [_facade(rng, extent, 20.0, 5.0, 30.0, 5.0, 30.0) for _ in range(n_facades)]
    edges = [e for q in quads for e in _facade_edges(q)]
    types = np.array([QUAD] * n_facades + [EDGE] * len(edges), dtype=np.uint8)
    verts = np.array(quads + edges)
    tx = np.array([[extent / 2, extent / 2, 10.0]])
    c = (np.arange(rx_grid) + 0.5) * (extent / rx_grid)
    gx, gy = np.meshgrid(c, c, indexing="ij")
    rx = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 1.5)], axis=1)
    qa = rng.choice(n_facades, size=n_alpha_quads, replace=False)
    # candidate diffraction edges: top (1), left (2), right (3) of every facade
    cand = np.array([n_facades + 4 * f + k for f in range(n_facades) for k in (1, 2, 3)])
    ea = rng.choice(cand, size=n_alpha_edges, replace=False)
    alphabet = np.sort(np.concatenate([qa, ea])).astype(np.int32)
    return Scene(types, verts, tx, rx, alphabet)


def city(seed: int = 0, n_obj: int = 256, quad_frac: float = 0.6, extent: float = 500.0,
         height: float = 60.0, n_tx: int = 1, n_rx: int = 16) -> Scene:
    """Random city block: vertical facades (5-30 m wide, up to 60 m high) and their edges."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_q = int(round(quad_frac * n_obj))
    quads = [_facade(rng, extent, 25.0, 5.0, 30.0, 5.0, height) for _ in range(n_q)]
    edges = []
    while len(edges) < n_obj - n_q:
        q = quads[int(rng.integers(0, n_q))]
        edges.append(_facade_edges(q)[int(rng.integers(1, 4))])
    types = np.array([QUAD] * n_q + [EDGE] * len(edges), dtype=np.uint8)
    verts = np.array(quads + edges)
    tx = np.column_stack([rng.uniform(100, 400, n_tx), rng.uniform(100, 400, n_tx), np.full(n_tx, 30.0)])
    rx = np.column_stack([rng.uniform(0, extent, n_rx), rng.uniform(0, extent, n_rx), np.full(n_rx, 1.5)])
    return Scene(types, verts, tx, rx)


def cotangents(seed: int, n_paths: int, n_max: int) -> tuple[np.ndarray, np.ndarray]:
    """Seeded per-path cotangents (dX [N, n_max, 3], dL [N]) for gradient checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dX = rng.standard_normal((n_paths, n_max, 3))
    dL = rng.standard_normal(n_paths)
    return dX, dL
