"""FP64 CPU oracle for the batched Fermat path solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it, and the two share no code: the oracle is a
plain C program (``fermat_oracle.c``) compiled with gcc and loaded here with
ctypes; the helpers below only marshal arrays and do plain sums.

Pins (see ``tests/test_oracle_pins.py``): image-method closed forms for
reflections, Keller's diffraction cone law and the unfolding closed form for a
single edge, brute-force grid search on order <= 2, stationarity of the
returned points, reversal symmetry, reparameterisation invariance, central
finite differences of the solve for the gradients, and ``itertools.product``
for the enumeration order.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fermat_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libfermat_oracle.so")
_lock = threading.Lock()
_lib = None

# status bits (same meaning as the library's)
VALID, CONVERGED, SOLVED, FP64_USED, DEGENERATE, REPEAT, NONFINITE, INVALID_INPUT = 1, 2, 4, 8, 16, 32, 64, 128
QUAD, EDGE = 0, 1
NEWTON, BFGS = 0, 1
# a solution with a segment shorter than this (metres) is a kink of L: DEGENERATE
DEG_TOL = 1e-3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, pthreads)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _BfgsParams(C.Structure):
    _fields_ = [("max_iters", C.c_int), ("fp_iters", C.c_int), ("scale_h0", C.c_int), ("safeguard", C.c_int),
                ("alpha0_first", C.c_double), ("alpha0", C.c_double), ("tol_step", C.c_double),
                ("stop_len", C.c_double)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _Batch(C.Structure):
    _fields_ = [("K", C.c_int), ("types", C.POINTER(C.c_uint8)), ("verts", _dp),
                ("n_tx", C.c_int), ("n_rx", C.c_int), ("tx", _dp), ("rx", _dp),
                ("M", C.c_int64), ("n_max", C.c_int), ("ids", _ip), ("order", _ip), ("tx_idx", _ip), ("rx_idx", _ip),
                ("solver", C.c_int), ("max_iters", C.c_int), ("bfgs", _BfgsParams), ("solved_tol", C.c_double),
                ("deg_tol", C.c_double),
                ("T_start", _dp), ("T", _dp), ("X", _dp), ("L", _dp), ("rho", _dp), ("bdist", _dp),
                ("status", _ip), ("iters", _ip),
                ("dX", _dp), ("dL", _dp), ("dtheta", _dp), ("n_threads", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_exhaustive_per_pair.restype = C.c_uint64
            L.orc_exhaustive_per_pair.argtypes = [C.c_int, C.c_int, C.c_int]
            L.orc_exhaustive_decode.restype = C.c_int
            L.orc_exhaustive_decode.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, _ip]
            L.orc_seeded_decode.restype = C.c_int
            L.orc_seeded_decode.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_uint64, _ip]
            L.orc_draw.restype = C.c_uint64
            L.orc_draw.argtypes = [C.c_uint64, C.c_uint64, C.c_int]
            L.orc_decode_batch.restype = None
            L.orc_decode_batch.argtypes = [C.c_int, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, _ip,
                                           C.c_int64, C.POINTER(C.c_uint64), C.c_int, _ip, _ip, _ip, _ip]
            L.orc_solve_batch.restype = C.c_int
            L.orc_solve_batch.argtypes = [C.POINTER(_Batch)]
            L.orc_object_record.restype = C.c_int
            L.orc_object_record.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
            path_args = [C.c_int, _ip, _dp, _dp, _dp, _dp]
            L.orc_path_length.restype = C.c_double
            L.orc_path_length.argtypes = path_args + [_dp]
            L.orc_path_grad_hess.restype = C.c_int
            L.orc_path_grad_hess.argtypes = path_args + [_dp, _dp, _dp]
            L.orc_path_solve.restype = C.c_int
            L.orc_path_solve.argtypes = path_args + [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                                     C.c_int, C.c_double, C.c_double, _dp, _dp, C.POINTER(C.c_int)]
            L.orc_path_residual.restype = C.c_double
            L.orc_path_residual.argtypes = path_args + [_dp]
            L.orc_path_fixed_point.restype = C.c_double
            L.orc_path_fixed_point.argtypes = path_args + [_dp, _dp, C.c_double, C.c_int]
            L.orc_path_vjp.restype = C.c_int
            L.orc_path_vjp.argtypes = path_args + [_dp, _dp, C.c_double, _dp]
            _lib = L
    return _lib


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


# --------------------------------------------------------------------------
# single-path helpers (objects given directly as b, A)
# --------------------------------------------------------------------------
class Path:
    """One interaction sequence: types [n], b [n,3], cols [n,2,3], x0, xe."""

    def __init__(self, types, b, cols, x0, xe):
        self.types = np.ascontiguousarray(types, dtype=np.int32)
        self.b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1, 3)
        self.cols = np.ascontiguousarray(cols, dtype=np.float64).reshape(-1, 2, 3)
        self.x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(3)
        self.xe = np.ascontiguousarray(xe, dtype=np.float64).reshape(3)
        self.n = len(self.types)

    def _args(self):
        return (self.n, _p(self.types, C.c_int32), _p(self.b), _p(self.cols), _p(self.x0), _p(self.xe))

    def length(self, t):
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(self.n, 2)
        return lib().orc_path_length(*self._args(), _p(t))

    def grad_hess(self, t):
        """Gradient (2n) and Hessian (2n x 2n) in the unified d = 2 parameters."""
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(self.n, 2)
        g = np.zeros(2 * self.n)
        H = np.zeros((2 * self.n, 2 * self.n))
        rc = lib().orc_path_grad_hess(*self._args(), _p(t), _p(g), _p(H))
        if rc != 0:
            raise ValueError("degenerate segment")
        return g, H

    def solve(self, solver=NEWTON, max_iters=200, fp_iters=1, alpha0_first=1.0, alpha0=1.0, scale_h0=0,
              safeguard=1, tol_step=0.0, deg_tol=DEG_TOL):
        t = np.zeros((self.n, 2))
        rho = np.zeros(1)
        it = C.c_int(0)
        st = lib().orc_path_solve(*self._args(), solver, max_iters, fp_iters, alpha0_first, alpha0, scale_h0,
                                  safeguard, tol_step, deg_tol, _p(t), _p(rho), C.byref(it))
        return t, int(st), float(rho[0]), int(it.value)

    def residual(self, t):
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(self.n, 2)
        return lib().orc_path_residual(*self._args(), _p(t))

    def fixed_point_alpha(self, t, p, alpha0, fp_iters):
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(self.n, 2)
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(2 * self.n)
        return lib().orc_path_fixed_point(*self._args(), _p(t), _p(p), alpha0, fp_iters)

    def vjp(self, t, dX, dL):
        """Per-path parameter gradient (x0[3], xe[3], then b_i, col_i1, col_i2 per slot)."""
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(self.n, 2)
        dX = np.ascontiguousarray(dX, dtype=np.float64).reshape(self.n, 3)
        out = np.zeros(6 + 9 * self.n)
        rc = lib().orc_path_vjp(*self._args(), _p(t), _p(dX), float(dL), _p(out))
        if rc != 0:
            raise ValueError(f"vjp failed ({rc})")
        return out

    def points(self, t):
        t = np.asarray(t, dtype=np.float64).reshape(self.n, 2)
        return self.b + np.einsum("nkc,nk->nc", self.cols, t)


def object_record(obj_type: int, verts: np.ndarray):
    v = np.ascontiguousarray(verts, dtype=np.float64).reshape(9)
    b, a1, a2 = np.zeros(3), np.zeros(3), np.zeros(3)
    rc = lib().orc_object_record(int(obj_type), _p(v), _p(b), _p(a1), _p(a2))
    if rc != 0:
        raise ValueError(f"degenerate object ({rc})")
    return b, np.stack([a1, a2])


def path_from_scene(scene, ids, tx_i=0, rx_i=0) -> Path:
    recs = [object_record(scene.types[o], scene.verts[o]) for o in ids]
    return Path([scene.types[o] for o in ids], [r[0] for r in recs], [r[1] for r in recs],
                scene.tx[tx_i], scene.rx[rx_i])


# --------------------------------------------------------------------------
# enumeration (Sec. III: all ordered sequences of n objects, n = lo..hi)
# --------------------------------------------------------------------------
def exhaustive_per_pair(K: int, lo: int, hi: int) -> int:
    return int(lib().orc_exhaustive_per_pair(K, lo, hi))


def _decode(scene, mode, seed, lo, hi, per_pair, g):
    g = np.ascontiguousarray(g, dtype=np.uint64)
    M = len(g)
    ids = np.empty((M, hi), dtype=np.int32)
    order = np.empty(M, dtype=np.int32)
    ti = np.empty(M, dtype=np.int32)
    ri = np.empty(M, dtype=np.int32)
    alpha = np.ascontiguousarray(scene.alphabet, dtype=np.int32)
    lib().orc_decode_batch(mode, int(seed), len(alpha), lo, hi, int(per_pair), len(scene.rx), _p(alpha, C.c_int32), M,
                           g.ctypes.data_as(C.POINTER(C.c_uint64)), hi, _p(ids, C.c_int32), _p(order, C.c_int32),
                           _p(ti, C.c_int32), _p(ri, C.c_int32))
    return ids, order, ti, ri


def exhaustive_paths(scene, lo: int, hi: int, g=None):
    """Decode global indices g of an exhaustive batch into (ids, order, tx_idx, rx_idx).

    g = ((tx * n_rx) + rx) * per_pair + r; r enumerates orders lo..hi, each in
    itertools.product order over the alphabet.
    """
    spp = exhaustive_per_pair(len(scene.alphabet), lo, hi)
    if g is None:
        g = np.arange(spp * len(scene.tx) * len(scene.rx), dtype=np.uint64)
    return _decode(scene, 0, 0, lo, hi, spp, g)


def seeded_paths(scene, seed: int, per_pair: int, lo: int, hi: int, g=None):
    """Decode a seeded batch: per_pair sequences for each TX/RX pair, drawn by splitmix64."""
    if g is None:
        g = np.arange(per_pair * len(scene.tx) * len(scene.rx), dtype=np.uint64)
    return _decode(scene, 1, seed, lo, hi, per_pair, g)


# --------------------------------------------------------------------------
# batch solve / backward
# --------------------------------------------------------------------------
def solve(scene, ids, order, tx_idx, rx_idx, solver=NEWTON, max_iters=200, fp_iters=1, alpha0_first=1.0,
          alpha0=1.0, scale_h0=0, safeguard=1, tol_step=0.0, stop_len=0.0, solved_tol=1e-5, deg_tol=DEG_TOL,
          n_threads=None, dX=None, dL=None, T_start=None):
    """Solve every listed path; returns a dict of numpy arrays (and 'dtheta' if cotangents are given)."""
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    M, n_max = ids.shape
    order = np.ascontiguousarray(order, dtype=np.int32)
    tx_idx = np.ascontiguousarray(tx_idx, dtype=np.int32)
    rx_idx = np.ascontiguousarray(rx_idx, dtype=np.int32)
    out = {"T": np.zeros((M, n_max, 2)), "X": np.zeros((M, n_max, 3)), "L": np.zeros(M), "rho": np.zeros(M),
           "bdist": np.zeros(M), "status": np.zeros(M, dtype=np.int32), "iters": np.zeros(M, dtype=np.int32)}
    B = _Batch()
    B.K = scene.n_obj
    B.types = _p(scene.types, C.c_uint8)
    B.verts = _p(scene.verts)
    B.n_tx, B.n_rx = len(scene.tx), len(scene.rx)
    B.tx, B.rx = _p(scene.tx), _p(scene.rx)
    B.M, B.n_max = M, n_max
    B.ids, B.order, B.tx_idx, B.rx_idx = (_p(a, C.c_int32) for a in (ids, order, tx_idx, rx_idx))
    B.solver, B.max_iters = solver, max_iters
    B.bfgs = _BfgsParams(max_iters, fp_iters, scale_h0, safeguard, alpha0_first, alpha0, tol_step, stop_len)
    B.solved_tol = solved_tol
    B.deg_tol = deg_tol
    Ts = None if T_start is None else np.ascontiguousarray(T_start, dtype=np.float64).reshape(M, n_max, 2)
    B.T_start = _p(Ts)
    B.T, B.X, B.L, B.rho, B.bdist = (_p(out[k]) for k in ("T", "X", "L", "rho", "bdist"))
    B.status, B.iters = _p(out["status"], C.c_int32), _p(out["iters"], C.c_int32)
    keep = []
    if dX is not None or dL is not None:
        dXa = np.ascontiguousarray(dX if dX is not None else np.zeros((M, n_max, 3)), dtype=np.float64)
        dLa = np.ascontiguousarray(dL if dL is not None else np.zeros(M), dtype=np.float64)
        out["dtheta"] = np.zeros((M, 6 + 9 * n_max))
        B.dX, B.dL, B.dtheta = _p(dXa), _p(dLa), _p(out["dtheta"])
        keep += [dXa, dLa]
    B.n_threads = int(n_threads or os.cpu_count() or 1)
    lib().orc_solve_batch(C.byref(B))
    return out


def reduce_gradients(scene, ids, order, tx_idx, rx_idx, dtheta):
    """Sum per-path parameter gradients into TX, RX and vertex gradients.

    Vertex chain rule: a plane (v0, v1, v3) has b = v0, a1 = v1 - v0,
    a2 = v3 - v0; an edge (e0, e1) has b = e0, a1 = e1 - e0.
    """
    K = scene.n_obj
    g_tx = np.zeros((len(scene.tx), 3))
    g_rx = np.zeros((len(scene.rx), 3))
    g_obj = np.zeros((K, 3, 3))  # (b, a1, a2)
    order = np.asarray(order)
    dtheta = np.asarray(dtheta, dtype=np.float64)
    # plain sums over paths (np.add.at adds repeated indices one by one)
    np.add.at(g_tx, np.asarray(tx_idx), dtheta[:, 0:3])
    np.add.at(g_rx, np.asarray(rx_idx), dtheta[:, 3:6])
    for i in range(ids.shape[1]):
        on = order > i
        np.add.at(g_obj, np.asarray(ids)[on, i], dtheta[on, 6 + 9 * i: 15 + 9 * i].reshape(-1, 3, 3))
    g_vert = np.zeros((K, 3, 3))
    gb, ga1, ga2 = g_obj[:, 0], g_obj[:, 1], g_obj[:, 2]
    quad = scene.types == QUAD
    g_vert[:, 0] = gb - ga1 - np.where(quad[:, None], ga2, 0.0)
    g_vert[:, 1] = ga1
    g_vert[:, 2] = np.where(quad[:, None], ga2, 0.0)
    return g_tx, g_rx, g_vert
