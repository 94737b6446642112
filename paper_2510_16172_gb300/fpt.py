"""Thin Python binding of the C ABI in include/fpt.h (argument marshalling only).

Every computation runs in the CUDA library ``libfpt.so``; this module loads
it with ctypes, passes raw pointers of torch CUDA tensors and numpy host
arrays, and raises on non-zero status.  There is no CPU fallback: if the
library is missing, importing the functions raises ``FptLibraryMissing``.

The functions keep the C names without the ``fpt_`` prefix:
``create / destroy / set_stream / sync / scene_upload / scene_free /
set_endpoints / batch_exhaustive / batch_seeded / batch_explicit /
batch_size / batch_free / enumerate / solve / validity / backward /
count_status``.  ``Context``, ``Scene`` and ``Batch`` wrap the handles.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfpt.so")

# status bits (include/fpt.h)
ST_VALID, ST_CONVERGED, ST_SOLVED, ST_FP64, ST_DEGENERATE, ST_REPEAT, ST_NONFINITE, ST_INVALID_INPUT = (
    1, 2, 4, 8, 16, 32, 64, 128)
QUAD, EDGE = 0, 1
_ERRORS = {1: "FPT_EINVAL", 2: "FPT_ENOMEM", 3: "FPT_ECUDA", 4: "FPT_EDEVICE", 5: "FPT_EUNSUPPORTED"}


class FptLibraryMissing(RuntimeError):
    pass


class FptError(RuntimeError):
    pass


class SolveParams(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("fp_iters", C.c_int32), ("polish", C.c_int32), ("fixed_iters", C.c_int32),
                ("tol_step", C.c_float), ("solved_tol", C.c_float), ("deg_tol", C.c_float), ("cond_fp64", C.c_float),
                ("init_mode", C.c_int32), ("polish_fp64", C.c_int32), ("refill", C.c_int32),
                ("specialize", C.c_int32), ("fuse_adjoint", C.c_int32),
                ("kink_stop", C.c_float), ("polish_all", C.c_int32), ("polish_radius", C.c_float),
                ("reserved", C.c_int32 * 4)]


class TrainParams(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("lr_decay", C.c_float),
                ("seed", C.c_uint64), ("reserved", C.c_int32 * 4)]


# every symbol declared in include/fpt.h with (restype, argtypes)
_vp = C.c_void_p
_SIGS = {
    "fpt_default_params": (None, [C.POINTER(SolveParams)]),
    "fpt_create": (C.c_int, [C.POINTER(_vp), C.c_int, _vp]),
    "fpt_destroy": (None, [_vp]),
    "fpt_set_stream": (C.c_int, [_vp, _vp]),
    "fpt_last_error": (C.c_char_p, [_vp]),
    "fpt_set_accumulation": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "fpt_backward_dropped": (C.c_int, [_vp, C.POINTER(C.c_uint64)]),
    "fpt_sync": (C.c_int, [_vp]),
    "fpt_scene_upload": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.POINTER(_vp)]),
    "fpt_scene_free": (None, [_vp]),
    "fpt_scene_upload_device": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp, C.POINTER(_vp)]),
    "fpt_set_endpoints": (C.c_int, [_vp, _vp, C.c_int32, _vp, C.c_int32]),
    "fpt_set_endpoints_device": (C.c_int, [_vp, _vp, C.c_int32, _vp, C.c_int32]),
    "fpt_scene_update_vertices": (C.c_int, [_vp, _vp]),
    "fpt_batch_exhaustive": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32, C.POINTER(_vp)]),
    "fpt_batch_seeded": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_uint64, C.c_uint64, C.c_int32, C.c_int32,
                                   C.POINTER(_vp)]),
    "fpt_batch_explicit": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_uint64, C.c_int32, C.POINTER(_vp)]),
    "fpt_batch_size": (C.c_int, [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_int32)]),
    "fpt_batch_free": (None, [_vp]),
    "fpt_enumerate": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "fpt_solve": (C.c_int, [_vp, _vp, _vp, C.POINTER(SolveParams), _vp, _vp, _vp, _vp, _vp, _vp]),
    "fpt_validity": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fpt_backward": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_uint8, _vp, _vp, _vp]),
    "fpt_solve_grad": (C.c_int, [_vp, _vp, _vp, C.POINTER(SolveParams), _vp, _vp, C.c_uint8, _vp, _vp, _vp, _vp, _vp,
                                 _vp, _vp, _vp, _vp]),
    "fpt_count_status": (C.c_int, [_vp, _vp, C.c_uint64, C.c_uint8, C.POINTER(C.c_uint64)]),
    "fpt_backward_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_uint8, _vp, _vp, _vp]),
    "fpt_occlusion": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_uint8, C.c_float, _vp]),
    "fpt_backward_unrolled": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fpt_tc_gemm_bf16": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp]),
    "fpt_mlp_create": (C.c_int, [_vp, C.c_uint64, C.c_float, C.POINTER(_vp)]),
    "fpt_mlp_free": (None, [_vp]),
    "fpt_mlp_get_params": (C.c_int, [_vp, _vp]),
    "fpt_mlp_set_params": (C.c_int, [_vp, _vp]),
    "fpt_mlp_save": (C.c_int, [_vp, C.c_char_p]),
    "fpt_mlp_load": (C.c_int, [_vp, C.c_char_p, C.POINTER(_vp)]),
    "fpt_mlp_features": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "fpt_mlp_forward": (C.c_int, [_vp, _vp, _vp, C.c_uint64, _vp]),
    "fpt_mlp_loss_grad": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_uint64, C.POINTER(C.c_float), _vp]),
    "fpt_mlp_train_step": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_uint64, C.c_float, C.POINTER(C.c_float)]),
    "fpt_mlp_train": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_uint64, C.POINTER(TrainParams), _vp]),
    "fpt_mlp_infer": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "fpt_set_init_mlp": (C.c_int, [_vp, _vp]),
    "fpt_check_bounded_wait": (C.c_int, [_vp, C.c_uint32, C.c_int, C.POINTER(C.c_uint64)]),
    "fpt_profile_enable": (C.c_int, [_vp, C.c_int]),
    "fpt_profile_read": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.c_int]),
}
K_BFGS, K_POLISH, K_BACKWARD, K_OTHER, K_MLP, K_COUNT = 0, 1, 2, 3, 4, 5

_lock = threading.Lock()
_lib = None


def library(path: str | None = None):
    """Load libfpt.so (built by paper_2510_16172_gb300.build); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise FptLibraryMissing(f"{p} not found: run paper_2510_16172_gb300.build.build() first")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def default_params(**overrides) -> SolveParams:
    p = SolveParams()
    library().fpt_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _ptr(x):
    """Raw pointer of a torch tensor / numpy array, or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _check(ctx_handle, rc):
    if rc != 0:
        msg = library().fpt_last_error(ctx_handle)
        raise FptError(f"{_ERRORS.get(rc, rc)}: {msg.decode() if msg else ''}")


def _is_cuda_tensor(x) -> bool:
    return getattr(x, "is_cuda", False) is True


def _need_cuda(t, dtype, name):
    import torch

    if t is None:
        return
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise FptError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
class Context:
    """fpt_create / fpt_destroy; launches on the given stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.stream = stream
        h = _vp()
        rc = library().fpt_create(C.byref(h), device, _vp(stream.cuda_stream))
        if rc != 0:
            raise FptError(f"fpt_create failed ({_ERRORS.get(rc, rc)})")
        self.handle = h

    def set_stream(self, stream):
        self.stream = stream
        _check(self.handle, library().fpt_set_stream(self.handle, _vp(stream.cuda_stream)))

    def sync(self):
        _check(self.handle, library().fpt_sync(self.handle))

    def set_accumulation(self, flush_tiles: int = 64, smem: int = 1):
        """fpt_set_accumulation: how the backward calls sum the per-path gradient terms."""
        _check(self.handle, library().fpt_set_accumulation(self.handle, int(flush_tiles), int(smem)))

    def close(self):
        if getattr(self, "handle", None):
            library().fpt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """fpt_scene_upload + fpt_set_endpoints (host float64 inputs)."""

    def __init__(self, ctx: Context, types, verts, tx=None, rx=None, centre=None):
        """Host float64 vertices: fpt_scene_upload.  A CUDA float32 tensor [n_obj, 3, 3]:
        fpt_scene_upload_device, recentred on `centre` (host, 3 floats; None = origin)."""
        self.ctx = ctx
        self.types = np.ascontiguousarray(types, dtype=np.uint8)
        h = _vp()
        if _is_cuda_tensor(verts):
            import torch

            _need_cuda(verts, torch.float32, "verts")
            if verts.numel() != 9 * len(self.types):
                raise FptError("verts must be [n_obj, 3, 3]")
            self.verts = verts
            c = None if centre is None else np.ascontiguousarray(centre, dtype=np.float64).reshape(3)
            _check(ctx.handle, library().fpt_scene_upload_device(ctx.handle, _ptr(self.types), _ptr(verts),
                                                                 len(self.types), _ptr(c), C.byref(h)))
        else:
            self.verts = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, 3, 3)
            _check(ctx.handle, library().fpt_scene_upload(ctx.handle, _ptr(self.types), _ptr(self.verts),
                                                          len(self.types), C.byref(h)))
        self.handle = h
        self.n_tx = self.n_rx = 0
        if tx is not None:
            self.set_endpoints(tx, rx)

    @property
    def n_obj(self):
        return len(self.types)

    def set_endpoints(self, tx, rx):
        """Host float64 arrays: fpt_set_endpoints.  CUDA float32 tensors [n, 3]: fpt_set_endpoints_device
        (the records are built on the device; the tensors are read when the stream reaches the call)."""
        if _is_cuda_tensor(tx) or _is_cuda_tensor(rx):
            import torch

            _need_cuda(tx, torch.float32, "tx")
            _need_cuda(rx, torch.float32, "rx")
            if tx.dim() != 2 or tx.shape[1] != 3 or rx.dim() != 2 or rx.shape[1] != 3:
                raise FptError("tx and rx must be [n, 3]")
            _check(self.ctx.handle, library().fpt_set_endpoints_device(self.handle, _ptr(tx), tx.shape[0], _ptr(rx),
                                                                       rx.shape[0]))
            self.n_tx, self.n_rx = int(tx.shape[0]), int(rx.shape[0])
            return
        tx = np.ascontiguousarray(np.atleast_2d(tx), dtype=np.float64)
        rx = np.ascontiguousarray(np.atleast_2d(rx), dtype=np.float64)
        _check(self.ctx.handle, library().fpt_set_endpoints(self.handle, _ptr(tx), len(tx), _ptr(rx), len(rx)))
        self.n_tx, self.n_rx = len(tx), len(rx)

    def update_vertices(self, verts):
        """fpt_scene_update_vertices from a CUDA float32 tensor [n_obj, 3, 3] (types and centre unchanged)."""
        import torch

        _need_cuda(verts, torch.float32, "verts")
        if verts.numel() != 9 * self.n_obj:
            raise FptError("verts must be [n_obj, 3, 3]")
        _check(self.ctx.handle, library().fpt_scene_update_vertices(self.handle, _ptr(verts)))

    def close(self):
        if getattr(self, "handle", None):
            library().fpt_scene_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A candidate-sequence batch: exhaustive, seeded or explicit."""

    def __init__(self, ctx: Context, handle, keep=()):
        self.ctx = ctx
        self.handle = handle
        self._keep = keep
        n = C.c_uint64(0)
        m = C.c_int32(0)
        _check(ctx.handle, library().fpt_batch_size(handle, C.byref(n), C.byref(m)))
        self.n_paths, self.n_max = int(n.value), int(m.value)

    @classmethod
    def exhaustive(cls, ctx, scene, order_lo, order_hi, alphabet=None):
        a = None if alphabet is None else np.ascontiguousarray(alphabet, dtype=np.int32)
        h = _vp()
        _check(ctx.handle, library().fpt_batch_exhaustive(ctx.handle, scene.handle, _ptr(a), 0 if a is None else len(a),
                                                          order_lo, order_hi, C.byref(h)))
        return cls(ctx, h)

    @classmethod
    def seeded(cls, ctx, scene, seed, per_pair, order_lo, order_hi, alphabet=None):
        a = None if alphabet is None else np.ascontiguousarray(alphabet, dtype=np.int32)
        h = _vp()
        _check(ctx.handle, library().fpt_batch_seeded(ctx.handle, scene.handle, _ptr(a), 0 if a is None else len(a),
                                                      int(seed), int(per_pair), order_lo, order_hi, C.byref(h)))
        return cls(ctx, h)

    @classmethod
    def explicit(cls, ctx, scene, ids, order, tx_idx, rx_idx):
        import torch

        _need_cuda(ids, torch.int32, "ids")
        _need_cuda(order, torch.uint8, "order")
        _need_cuda(tx_idx, torch.int32, "tx_idx")
        _need_cuda(rx_idx, torch.int32, "rx_idx")
        h = _vp()
        _check(ctx.handle, library().fpt_batch_explicit(ctx.handle, scene.handle, _ptr(ids), _ptr(order), _ptr(tx_idx),
                                                        _ptr(rx_idx), ids.shape[0], ids.shape[1], C.byref(h)))
        return cls(ctx, h, keep=(ids, order, tx_idx, rx_idx))

    def close(self):
        if getattr(self, "handle", None):
            library().fpt_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# calls (outputs are torch CUDA tensors on the context's device)
# ---------------------------------------------------------------------------
def enumerate(ctx: Context, batch: Batch):
    import torch

    dev = torch.device("cuda", ctx.device)
    N, m = batch.n_paths, batch.n_max
    ids = torch.empty((N, m), dtype=torch.int32, device=dev)
    order = torch.empty(N, dtype=torch.uint8, device=dev)
    txi = torch.empty(N, dtype=torch.int32, device=dev)
    rxi = torch.empty(N, dtype=torch.int32, device=dev)
    _check(ctx.handle, library().fpt_enumerate(ctx.handle, batch.handle, _ptr(ids), _ptr(order), _ptr(txi), _ptr(rxi)))
    return ids, order, txi, rxi


def alloc_outputs(ctx: Context, batch: Batch, with_X=True, with_rho=True, with_iters=True):
    import torch

    dev = torch.device("cuda", ctx.device)
    N, m = batch.n_paths, batch.n_max
    return {
        "T": torch.empty((N, m, 2), dtype=torch.float32, device=dev),
        "X": torch.empty((N, m, 3), dtype=torch.float32, device=dev) if with_X else None,
        "L": torch.empty(N, dtype=torch.float32, device=dev),
        "status": torch.empty(N, dtype=torch.uint8, device=dev),
        "iters": torch.empty(N, dtype=torch.uint8, device=dev) if with_iters else None,
        "rho": torch.empty(N, dtype=torch.float32, device=dev) if with_rho else None,
    }


def solve(ctx: Context, scene: Scene, batch: Batch, params: SolveParams | None = None, out=None):
    """fpt_solve; returns the dict of output tensors (T, X, L, status, iters, rho)."""
    import torch

    out = out if out is not None else alloc_outputs(ctx, batch)
    for k, dt in (("T", torch.float32), ("X", torch.float32), ("L", torch.float32), ("status", torch.uint8),
                  ("iters", torch.uint8), ("rho", torch.float32)):
        _need_cuda(out.get(k), dt, k)
    p = params if params is not None else default_params()
    _check(ctx.handle, library().fpt_solve(ctx.handle, scene.handle, batch.handle, C.byref(p), _ptr(out["T"]),
                                           _ptr(out.get("X")), _ptr(out.get("L")), _ptr(out["status"]),
                                           _ptr(out.get("iters")), _ptr(out.get("rho"))))
    return out


def solve_grad(ctx: Context, scene: Scene, batch: Batch, params: SolveParams | None = None, dX=None, dL=None,
               dL_status_mask=0, out=None, grads=None):
    """fpt_solve_grad: the outputs of solve() and the gradients of backward() in one pass.

    Returns (out dict, (g_tx, g_rx, g_vertices)).
    """
    import torch

    out = out if out is not None else alloc_outputs(ctx, batch)
    for k, dt in (("T", torch.float32), ("X", torch.float32), ("L", torch.float32), ("status", torch.uint8),
                  ("iters", torch.uint8), ("rho", torch.float32)):
        _need_cuda(out.get(k), dt, k)
    _need_cuda(dX, torch.float32, "dX")
    _need_cuda(dL, torch.float32, "dL")
    dev = out["T"].device
    if grads is None:
        grads = (torch.empty((scene.n_tx, 3), dtype=torch.float32, device=dev),
                 torch.empty((scene.n_rx, 3), dtype=torch.float32, device=dev),
                 torch.empty((scene.n_obj, 3, 3), dtype=torch.float32, device=dev))
    g_tx, g_rx, g_v = grads
    p = params if params is not None else default_params()
    _check(ctx.handle, library().fpt_solve_grad(ctx.handle, scene.handle, batch.handle, C.byref(p), _ptr(dX),
                                                _ptr(dL), int(dL_status_mask), _ptr(out["T"]), _ptr(out.get("X")),
                                                _ptr(out.get("L")), _ptr(out["status"]), _ptr(out.get("iters")),
                                                _ptr(out.get("rho")), _ptr(g_tx), _ptr(g_rx), _ptr(g_v)))
    return out, grads


def validity(ctx: Context, scene: Scene, batch: Batch, T):
    """fpt_validity at caller-given T; returns (mask, bdist, rho)."""
    import torch

    _need_cuda(T, torch.float32, "T")
    dev = T.device
    N = batch.n_paths
    mask = torch.empty(N, dtype=torch.uint8, device=dev)
    bd = torch.empty(N, dtype=torch.float32, device=dev)
    rho = torch.empty(N, dtype=torch.float32, device=dev)
    _check(ctx.handle, library().fpt_validity(ctx.handle, scene.handle, batch.handle, _ptr(T), _ptr(mask), _ptr(bd),
                                              _ptr(rho)))
    return mask, bd, rho


def backward(ctx: Context, scene: Scene, batch: Batch, T, status=None, dX=None, dL=None, dL_status_mask=0, out=None):
    """fpt_backward; returns (g_tx [n_tx,3], g_rx [n_rx,3], g_vertices [n_obj,3,3])."""
    import torch

    _need_cuda(T, torch.float32, "T")
    _need_cuda(status, torch.uint8, "status")
    _need_cuda(dX, torch.float32, "dX")
    _need_cuda(dL, torch.float32, "dL")
    dev = T.device
    if out is None:
        out = (torch.empty((scene.n_tx, 3), dtype=torch.float32, device=dev),
               torch.empty((scene.n_rx, 3), dtype=torch.float32, device=dev),
               torch.empty((scene.n_obj, 3, 3), dtype=torch.float32, device=dev))
    g_tx, g_rx, g_v = out
    _check(ctx.handle, library().fpt_backward(ctx.handle, scene.handle, batch.handle, _ptr(T), _ptr(status), _ptr(dX),
                                              _ptr(dL), int(dL_status_mask), _ptr(g_tx), _ptr(g_rx), _ptr(g_v)))
    return g_tx, g_rx, g_v


def backward_noalloc(ctx: Context, scene: Scene, batch: Batch, T, status=None, dX=None, dL=None, dL_status_mask=0,
                     out=None):
    """fpt_backward_noalloc: same results as backward(), scratch in the library's fixed array.

    The output tensors must be supplied (out = (g_tx, g_rx, g_vertices)) by
    callers that cannot allocate; when out is None they are created here.
    """
    import torch

    _need_cuda(T, torch.float32, "T")
    _need_cuda(status, torch.uint8, "status")
    _need_cuda(dX, torch.float32, "dX")
    _need_cuda(dL, torch.float32, "dL")
    dev = T.device
    if out is None:
        out = (torch.empty((scene.n_tx, 3), dtype=torch.float32, device=dev),
               torch.empty((scene.n_rx, 3), dtype=torch.float32, device=dev),
               torch.empty((scene.n_obj, 3, 3), dtype=torch.float32, device=dev))
    g_tx, g_rx, g_v = out
    _check(ctx.handle, library().fpt_backward_noalloc(ctx.handle, scene.handle, batch.handle, _ptr(T), _ptr(status),
                                                      _ptr(dX), _ptr(dL), int(dL_status_mask), _ptr(g_tx),
                                                      _ptr(g_rx), _ptr(g_v)))
    return g_tx, g_rx, g_v


def occlusion(ctx: Context, scene: Scene, batch: Batch, T, status=None, status_mask: int = 0, tol: float = 0.0,
              out=None):
    """fpt_occlusion: per path an int16 bit mask, bit j set when segment j is obstructed."""
    import torch

    _need_cuda(T, torch.float32, "T")
    _need_cuda(status, torch.uint8, "status")
    if out is None:
        out = torch.zeros(batch.n_paths, dtype=torch.int16, device=T.device)
    _need_cuda(out, torch.int16, "out")
    if out.numel() != batch.n_paths or T.numel() != batch.n_paths * batch.n_max * 2:
        raise FptError("T must be [N, n_max, 2] and out [N] for the batch")
    if status is not None and status.numel() != batch.n_paths:
        raise FptError("status must be [N]")
    _check(ctx.handle, library().fpt_occlusion(ctx.handle, scene.handle, batch.handle, _ptr(T), _ptr(status),
                                               int(status_mask), float(tol), _ptr(out)))
    return out


def backward_unrolled(ctx: Context, scene: Scene, batch: Batch, steps: int, fp_iters: int = 1, dX=None, dL=None,
                      want_T: bool = False, out=None):
    """fpt_backward_unrolled: gradient through `steps` solver steps by reverse mode.

    Returns (g_tx, g_rx, g_vertices, T, status); T [N, n_max, 2] (the last
    iterate) only with want_T, status [N] always.
    """
    import torch

    _need_cuda(dX, torch.float32, "dX")
    _need_cuda(dL, torch.float32, "dL")
    dev = f"cuda:{ctx.device}"
    if out is None:
        out = (torch.empty((scene.n_tx, 3), dtype=torch.float32, device=dev),
               torch.empty((scene.n_rx, 3), dtype=torch.float32, device=dev),
               torch.empty((scene.n_obj, 3, 3), dtype=torch.float32, device=dev))
    g_tx, g_rx, g_v = out
    N = batch.n_paths
    T = torch.zeros((N, batch.n_max, 2), dtype=torch.float32, device=dev) if want_T else None
    status = torch.zeros(N, dtype=torch.uint8, device=dev)
    _check(ctx.handle, library().fpt_backward_unrolled(ctx.handle, scene.handle, batch.handle, int(steps),
                                                       int(fp_iters), _ptr(dX), _ptr(dL), _ptr(T), _ptr(status),
                                                       _ptr(g_tx), _ptr(g_rx), _ptr(g_v)))
    return g_tx, g_rx, g_v, T, status


def profile_enable(ctx: Context, on: bool = True):
    _check(ctx.handle, library().fpt_profile_enable(ctx.handle, 1 if on else 0))


def profile_read(ctx: Context, reset: bool = True):
    """Summed device milliseconds and launch counts per kernel class (K_BFGS, K_POLISH, K_BACKWARD, K_OTHER)."""
    ms = (C.c_double * K_COUNT)()
    n = (C.c_uint64 * K_COUNT)()
    _check(ctx.handle, library().fpt_profile_read(ctx.handle, ms, n, 1 if reset else 0))
    return list(ms), list(n)


MLP_FEATURES, MLP_OUT, MLP_NPARAMS = 64, 16, 152336


class Mlp:
    """Warm-start network (fpt_mlp_*): create (seeded) or load, features, forward, loss/grad, Adam step."""

    def __init__(self, ctx: Context, seed: int = 0, length_scale: float = 10.0, handle=None):
        self.ctx = ctx
        if handle is None:
            h = _vp()
            _check(ctx.handle, library().fpt_mlp_create(ctx.handle, int(seed), float(length_scale), C.byref(h)))
            handle = h
        self.handle = handle

    @classmethod
    def load(cls, ctx: Context, path: str):
        h = _vp()
        _check(ctx.handle, library().fpt_mlp_load(ctx.handle, os.fsencode(path), C.byref(h)))
        return cls(ctx, handle=h)

    def save(self, path: str):
        _check(self.ctx.handle, library().fpt_mlp_save(self.handle, os.fsencode(path)))

    def get_params(self) -> np.ndarray:
        out = np.empty(MLP_NPARAMS, dtype=np.float32)
        _check(self.ctx.handle, library().fpt_mlp_get_params(self.handle, _ptr(out)))
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_NPARAMS:
            raise FptError("wrong parameter count")
        _check(self.ctx.handle, library().fpt_mlp_set_params(self.handle, _ptr(p)))

    def features(self, scene: Scene, batch: Batch, with_gram: bool = False):
        """Features [N, 64] (bf16), and with with_gram the loss's Gram matrices [N, 4, 3]."""
        import torch

        dev = f"cuda:{self.ctx.device}"
        X = torch.empty((batch.n_paths, MLP_FEATURES), dtype=torch.bfloat16, device=dev)
        G = torch.empty((batch.n_paths, 4, 3), dtype=torch.float32, device=dev) if with_gram else None
        _check(self.ctx.handle, library().fpt_mlp_features(self.ctx.handle, self.handle, scene.handle, batch.handle,
                                                           _ptr(X), _ptr(G)))
        return (X, G) if with_gram else X

    def forward(self, X):
        import torch

        _need_cuda(X, torch.bfloat16, "X")
        Y = torch.empty((X.shape[0], MLP_OUT), dtype=torch.float32, device=X.device)
        _check(self.ctx.handle, library().fpt_mlp_forward(self.ctx.handle, self.handle, _ptr(X), X.shape[0], _ptr(Y)))
        return Y

    def loss_grad(self, X, T, G):
        import torch

        _need_cuda(X, torch.bfloat16, "X")
        _need_cuda(T, torch.float32, "T")
        _need_cuda(G, torch.float32, "G")
        g = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=X.device)
        loss = C.c_float(0.0)
        _check(self.ctx.handle, library().fpt_mlp_loss_grad(self.ctx.handle, self.handle, _ptr(X), _ptr(T), _ptr(G),
                                                             X.shape[0], C.byref(loss), _ptr(g)))
        return float(loss.value), g

    def train_step(self, X, T, G, lr: float, want_loss: bool = True):
        import torch

        _need_cuda(X, torch.bfloat16, "X")
        _need_cuda(T, torch.float32, "T")
        _need_cuda(G, torch.float32, "G")
        loss = C.c_float(0.0)
        _check(self.ctx.handle, library().fpt_mlp_train_step(self.ctx.handle, self.handle, _ptr(X), _ptr(T), _ptr(G),
                                                              X.shape[0], float(lr),
                                                              C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def train(self, X, T, G, epochs: int, batch: int = 8192, lr: float = 1e-3, lr_decay: float = 0.5,
              seed: int = 0):
        """fpt_mlp_train: the whole schedule in the library (seeded shuffles, Adam steps); returns the
        per-epoch mean loss."""
        import torch

        _need_cuda(X, torch.bfloat16, "X")
        _need_cuda(T, torch.float32, "T")
        _need_cuda(G, torch.float32, "G")
        p = TrainParams(int(epochs), int(batch), float(lr), float(lr_decay), int(seed))
        hist = (C.c_float * int(epochs))()
        _check(self.ctx.handle, library().fpt_mlp_train(self.ctx.handle, self.handle, _ptr(X), _ptr(T), _ptr(G),
                                                         X.shape[0], C.byref(p), hist))
        return [float(v) for v in hist]

    def infer(self, scene: "Scene", batch: "Batch", out=None):
        """fpt_mlp_infer: the learned start T [N, n_max, 2] of every path of the batch."""
        import torch

        if out is None:
            out = torch.empty((batch.n_paths, batch.n_max, 2), dtype=torch.float32,
                              device=torch.device("cuda", self.ctx.device))
        _need_cuda(out, torch.float32, "out")
        _check(self.ctx.handle, library().fpt_mlp_infer(self.ctx.handle, self.handle, scene.handle, batch.handle,
                                                         _ptr(out)))
        return out

    def attach(self):
        """Use this network for fpt_solve with init_mode = 1."""
        _check(self.ctx.handle, library().fpt_set_init_mlp(self.ctx.handle, self.handle))

    def close(self):
        if getattr(self, "handle", None):
            library().fpt_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_gemm_bf16(ctx: Context, A, W, bias=None, out=None):
    """C = A W^T (+ bias) on the tensor cores; A [M,K], W [N,K] bf16 CUDA tensors."""
    import torch

    _need_cuda(A, torch.bfloat16, "A")
    _need_cuda(W, torch.bfloat16, "W")
    _need_cuda(bias, torch.float32, "bias")
    M, K = A.shape
    N = W.shape[0]
    if W.shape[1] != K:
        raise FptError("A and W disagree on K")
    C = out if out is not None else torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(ctx.handle, library().fpt_tc_gemm_bf16(ctx.handle, M, N, K, _ptr(A), _ptr(W), _ptr(bias), _ptr(C)))
    return C


def check_bounded_wait(ctx: Context, limit_us: int, arrive: bool) -> int:
    """fpt_check_bounded_wait: one CTA waits at most `limit_us` on an mbarrier that gets its arrival only
    if `arrive`; returns the wait's duration in ns.  Without the arrival the next ctx.sync() raises
    FptError (FPT_EDEVICE)."""
    ns = C.c_uint64(0)
    _check(ctx.handle, library().fpt_check_bounded_wait(ctx.handle, int(limit_us), 1 if arrive else 0, C.byref(ns)))
    return int(ns.value)


def backward_dropped(ctx: Context) -> int:
    """fpt_backward_dropped: paths of the last backward call left out as singular in FP64 too."""
    n = C.c_uint64(0)
    _check(ctx.handle, library().fpt_backward_dropped(ctx.handle, C.byref(n)))
    return int(n.value)


def count_status(ctx: Context, status, mask: int) -> int:
    import torch

    _need_cuda(status, torch.uint8, "status")
    n = C.c_uint64(0)
    _check(ctx.handle, library().fpt_count_status(ctx.handle, _ptr(status), status.numel(), mask, C.byref(n)))
    return int(n.value)
