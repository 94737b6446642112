"""Pins of the obstruction oracle (oracle/occlusion.py) against facts fixed outside it (CPU only):
hand-built cases, and an independent segment-triangle test (Moller-Trumbore on the two triangles of
each parallelogram) on random segments."""

import numpy as np

from oracle import occlusion
from paper_2510_16172_gb300 import scenes


def _scene(quads, tx, rx, edges=()):
    verts = [np.array(q, dtype=np.float64) for q in quads] + [np.array(e, dtype=np.float64) for e in edges]
    types = [scenes.QUAD] * len(quads) + [scenes.EDGE] * len(edges)
    return scenes.Scene(np.array(types), np.array(verts), np.atleast_2d(tx), np.atleast_2d(rx))


SQUARE = [[0, 0, 0], [1, 0, 0], [0, 1, 0]]  # v0, v1, v3 of the unit square in z = 0


def _masks(sc, ids, order, X):
    args = (sc, np.atleast_2d(ids), np.atleast_1d(order), [0] * len(np.atleast_1d(order)),
            [0] * len(np.atleast_1d(order)), np.asarray(X, dtype=np.float64).reshape(len(np.atleast_1d(order)), -1, 3))
    return occlusion.blocked_segments(*args), occlusion.decided(*args)


def test_hand_cases():
    # a direct path (order 0 is not a sequence: use a reflection elsewhere and look at its segments)
    wall = [[10, -5, -5], [10, 5, -5], [10, -5, 5]]  # the plane x = 10, a reflector far away
    sc = _scene([SQUARE, wall], [0.5, 0.5, 1.0], [0.5, 0.5, -1.0])
    # path TX -> point on the wall -> RX; segment 0 from (0.5, 0.5, 1) to (10, 0, 0) passes z = 0 at x ~ 5: outside
    m, _ = _masks(sc, [1], [1], [[10.0, 0.5, 0.0]])
    assert m[0] == 0
    # RX below the square, reflection point straight ahead: the second segment crosses z = 0 at (5.25, .5, 0)
    sc = _scene([SQUARE, wall], [0.5, 0.5, 1.0], [0.5, 0.5, -1.0])
    m, _ = _masks(sc, [1], [1], [[10.0, 0.5, 0.5]])
    assert m[0] == 0  # crossing at x ~ 5.2, outside the unit square
    # a path that bounces back over the square: TX (0.2, 0.5, 1) -> wall -> RX (0.8, 0.5, -1)
    sc = _scene([SQUARE, wall], [0.2, 0.5, 1.0], [0.8, 0.5, -1.0])
    # crossing of segment 1 from (10, .5, -0.9) to (0.8, .5, -1): never reaches z = 0 -> not blocked
    m, _ = _masks(sc, [1], [1], [[10.0, 0.5, -0.9]])
    assert m[0] == 0
    # segment 0 from (0.2, .5, 1) to (10, .5, -0.9) crosses z = 0 at x = 0.2 + 9.8 / 1.9 ~ 5.36: outside
    m, _ = _masks(sc, [1], [1], [[10.0, 0.5, -0.9]])
    assert m[0] == 0
    # now put the wall point low enough that segment 0 crosses z = 0 at x = 0.6, inside the square
    # (0.2, .5, 1) -> (10, .5, z): crossing at 0.2 + 9.8 / (1 - z) = 0.6  =>  z = 1 - 24.5
    m, sure = _masks(sc, [1], [1], [[10.0, 0.5, -23.5]])
    assert m[0] == 1 and sure[0]
    # an edge in the way blocks nothing
    sc2 = _scene([wall], [0.2, 0.5, 1.0], [0.8, 0.5, -1.0], edges=[[[0, 0.5, 0], [1, 0.5, 0], [0, 0, 0]]])
    m, _ = _masks(sc2, [0], [1], [[10.0, 0.5, -23.5]])
    assert m[0] == 0
    # the objects at a segment's ends never block it: reflect off the square itself
    sc3 = _scene([SQUARE], [0.2, 0.5, 1.0], [0.8, 0.5, 1.0])
    m, _ = _masks(sc3, [0], [1], [[0.5, 0.5, 0.0]])
    assert m[0] == 0
    # closed boundary: crossing exactly on the side u = 1 blocks
    sc4 = _scene([SQUARE, wall], [1.0, 0.5, 1.0], [0.8, 0.5, -1.0])
    m, sure = _masks(sc4, [1], [1], [[1.0, 0.5, -1.0]])  # segment 0 straight down through (1, .5, 0)
    assert m[0] == 1 and not sure[0]


def _moller_trumbore(P, Q, a, b, c):
    """Segment P->Q against triangle abc: (hit, s, barycentric u, v)."""
    d = Q - P
    e1, e2 = b - a, c - a
    h = np.cross(d, e2)
    det = e1 @ h
    if abs(det) < 1e-14:
        return False, None, None, None
    f = 1.0 / det
    sv = P - a
    u = f * (sv @ h)
    q = np.cross(sv, e1)
    v = f * (d @ q)
    s = f * (e2 @ q)
    return (u >= 0) and (v >= 0) and (u + v <= 1) and (0 <= s <= 1), s, u, v


def test_against_segment_triangle_intersection():
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(400):
        v0 = rng.uniform(-2, 2, 3)
        a1, a2 = rng.normal(size=3), rng.normal(size=3)
        quad = np.array([v0, v0 + a1, v0 + a2])
        wall = [[50, -5, -5], [50, 5, -5], [50, -5, 5]]  # the interaction object, far away
        P, R = rng.uniform(-4, 4, 3), rng.uniform(-4, 4, 3)
        sc = _scene([quad, wall], P, R)
        Xw = np.array([50.0, rng.uniform(-4, 4), rng.uniform(-4, 4)])
        m, sure = _masks(sc, [1], [1], [Xw])
        if not sure[0]:
            continue
        checked += 1
        for j, (A, B) in enumerate([(P, Xw), (Xw, R)]):
            hit1 = _moller_trumbore(A, B, v0, v0 + a1, v0 + a2)[0]
            hit2 = _moller_trumbore(A, B, v0 + a1 + a2, v0 + a2, v0 + a1)[0]
            assert bool((m[0] >> j) & 1) == (hit1 or hit2), (j, A, B, quad)
    assert checked > 300
