"""Geometry given as device FP32 arrays (fpt_scene_upload_device, fpt_scene_update_vertices,
fpt_set_endpoints_device): the records the kernels build equal the host upload's for the same
coordinates, so every solve is the same bit for bit; an endpoint sweep that replaces the RX ten
times with no synchronisation matches the oracle at every step; the autograd wrapper takes CUDA
tensors straight through; degenerate device geometry is reported through the error word.
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


def f32(sc):
    """The scene with every coordinate rounded to FP32 (what a device FP32 array holds)."""
    return scenes.Scene(sc.types, sc.verts.astype(np.float32).astype(np.float64),
                        sc.tx.astype(np.float32).astype(np.float64), sc.rx.astype(np.float32).astype(np.float64),
                        sc.alphabet)


def host_centre(verts, types):
    """The centre fpt_scene_upload takes: the middle of the bounding box of the used vertices."""
    used = np.concatenate([verts[k, :3 if t == scenes.QUAD else 2] for k, t in enumerate(types)])
    return 0.5 * (used.min(axis=0) + used.max(axis=0))


def run(ctx, scene, lo=1, hi=3, params=None):
    batch = fpt.Batch.exhaustive(ctx, scene, lo, hi)
    out = fpt.solve(ctx, scene, batch, params)
    return batch, out


def same(a, b):
    """Bit for bit (NaN where the other is NaN)."""
    import torch

    for k in ("T", "X", "L", "status", "iters", "rho"):
        x, y = a[k], b[k]
        if x.dtype.is_floating_point:
            assert torch.equal(x.isnan(), y.isnan()), k
            x, y = x.nan_to_num(nan=0.0), y.nan_to_num(nan=0.0)
        assert torch.equal(x, y), k


def test_device_scene_matches_host_scene_bit_for_bit(ctx):
    import torch

    sc = f32(scenes.tiny_scene(6, n_rx=3))
    host = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    _, ref = run(ctx, host)
    V = torch.as_tensor(sc.verts, dtype=torch.float32, device="cuda")
    tx = torch.as_tensor(sc.tx, dtype=torch.float32, device="cuda")
    rx = torch.as_tensor(sc.rx, dtype=torch.float32, device="cuda")
    dev = fpt.Scene(ctx, sc.types, V, tx, rx, centre=host_centre(sc.verts, sc.types))
    _, got = run(ctx, dev)
    ctx.sync()
    same(got, ref)
    # the obstruction test reads the occluder records: the same too
    b1 = fpt.Batch.exhaustive(ctx, host, 1, 3)
    b2 = fpt.Batch.exhaustive(ctx, dev, 1, 3)
    o1 = fpt.occlusion(ctx, host, b1, ref["T"], ref["status"], fpt.ST_VALID)
    o2 = fpt.occlusion(ctx, dev, b2, got["T"], got["status"], fpt.ST_VALID)
    ctx.sync()
    assert torch.equal(o1, o2)


def test_update_vertices_matches_a_fresh_scene(ctx):
    import torch

    a = f32(scenes.tiny_scene(7, n_rx=2))
    b = f32(scenes.tiny_scene(8, n_rx=2))
    scene = fpt.Scene(ctx, a.types, a.verts, a.tx, a.rx)
    centre = host_centre(a.verts, a.types)
    # b's objects with a's types: take b's vertices object by object where the types agree, a's elsewhere
    verts = np.where((a.types == b.types)[:, None, None], b.verts, a.verts)
    _, first = run(ctx, scene)
    first = {k: v.clone() for k, v in first.items() if v is not None}
    scene.update_vertices(torch.as_tensor(verts, dtype=torch.float32, device="cuda"))
    _, second = run(ctx, scene)
    ctx.sync()
    # a scene uploaded with these vertices and a's centre (device upload with that centre)
    ref_scene = fpt.Scene(ctx, a.types, torch.as_tensor(verts, dtype=torch.float32, device="cuda"),
                          torch.as_tensor(a.tx, dtype=torch.float32, device="cuda"),
                          torch.as_tensor(a.rx, dtype=torch.float32, device="cuda"), centre=centre)
    _, ref = run(ctx, ref_scene)
    _, ref_first = run(ctx, fpt.Scene(ctx, a.types, a.verts, a.tx, a.rx))
    ctx.sync()
    same(second, ref)
    same(first, ref_first)


def test_endpoint_sweep_without_synchronising_matches_the_oracle(ctx):
    """RX moved ten times through device arrays, each solve issued right after the update with no
    synchronisation; afterwards every step's points and lengths match the oracle for its RX."""
    import torch

    from test_gpu_parity import check_parity, oracle_solve

    sc = f32(scenes.tiny_scene(9, n_rx=2))
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 2)
    rng = np.random.default_rng(5)
    tx = torch.as_tensor(sc.tx, dtype=torch.float32, device="cuda")
    rx_all = rng.uniform(0.0, 10.0, (10, 2, 3)).astype(np.float32)
    rx_dev = torch.as_tensor(rx_all, device="cuda")
    outs = []
    for k in range(10):
        scene.set_endpoints(tx, rx_dev[k])
        outs.append(fpt.solve(ctx, scene, batch))
    ctx.sync()
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    for k in range(10):
        sk = scenes.Scene(sc.types, sc.verts, sc.tx, rx_all[k].astype(np.float64), sc.alphabet)
        ref = oracle_solve(sk, ids, order, ti, ri)
        g = {key: v.cpu().numpy() for key, v in outs[k].items() if v is not None}
        check_parity(g, ref)


def test_autograd_on_cuda_tensors_matches_oracle(ctx):
    """Gradients of a torch loss through FermatSolver with CUDA float32 inputs, against the oracle's VJP
    on the same (FP32) geometry; a second forward before the first backward does not change it."""
    import torch

    from paper_2510_16172_gb300.autograd import FermatSolver
    from test_gpu_parity import oracle_solve, regular

    sc = f32(scenes.tiny_scene(8, n_rx=2))
    solver = FermatSolver(sc.types, 1, 2, centre=host_centre(sc.verts, sc.types))
    tx = torch.tensor(sc.tx, dtype=torch.float32, device="cuda", requires_grad=True)
    rx = torch.tensor(sc.rx, dtype=torch.float32, device="cuda", requires_grad=True)
    verts = torch.tensor(sc.verts, dtype=torch.float32, device="cuda", requires_grad=True)
    X, L, status = solver(tx, rx, verts)
    # another forward on other geometry: the first backward must still use its own
    other = f32(scenes.tiny_scene(12, n_rx=2))
    solver(torch.as_tensor(other.tx, dtype=torch.float32, device="cuda"),
           torch.as_tensor(other.rx, dtype=torch.float32, device="cuda"),
           torch.as_tensor(np.where((sc.types == other.types)[:, None, None], other.verts, sc.verts),
                           dtype=torch.float32, device="cuda"))
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    ref = oracle_solve(sc, ids, order, ti, ri)
    keep = regular(ref["status"]) & (ref["minseg"] > 0.01)
    both = keep & ((status.cpu().numpy() & fpt.ST_SOLVED) > 0)
    assert both.sum() >= 0.98 * keep.sum()
    w, _ = scenes.cotangents(3, len(order), 2)
    wt = torch.as_tensor(w * both[:, None, None], dtype=torch.float32, device="cuda")
    valid = torch.as_tensor(((ref["status"] & oracle.VALID) > 0) & both, dtype=torch.float32, device="cuda")
    loss = (wt * X).sum() + (valid * L).sum()
    loss.backward()
    assert tx.grad.is_cuda and tx.grad.dtype == torch.float32
    e = oracle.solve(sc, ids, order, ti, ri, dX=w * both[:, None, None], dL=valid.double().cpu().numpy())
    e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, e["dtheta"])
    scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), 1.0)
    np.testing.assert_allclose(tx.grad.cpu().numpy(), e_tx, atol=2e-4 * scale)
    np.testing.assert_allclose(rx.grad.cpu().numpy(), e_rx, atol=2e-4 * scale)
    np.testing.assert_allclose(verts.grad.cpu().numpy(), e_v, atol=2e-4 * scale)


def test_degenerate_device_geometry_sets_the_error_word(ctx):
    import torch

    sc = f32(scenes.tiny_scene(2, n_rx=1))
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    ctx.sync()
    v = torch.as_tensor(sc.verts, dtype=torch.float32, device="cuda").clone()
    q = int(np.nonzero(sc.types == scenes.QUAD)[0][0])
    v[q, 2] = v[q, 0]  # v3 = v0: a zero-area plane
    scene.update_vertices(v)
    with pytest.raises(fpt.FptError, match="FPT_EDEVICE"):
        ctx.sync()
    ctx.sync()  # the word was cleared
    tx = torch.as_tensor(sc.tx, dtype=torch.float32, device="cuda")
    rx = torch.full((1, 3), float("nan"), dtype=torch.float32, device="cuda")
    scene.set_endpoints(tx, rx)
    with pytest.raises(fpt.FptError, match="FPT_EDEVICE"):
        ctx.sync()
    ctx.sync()
