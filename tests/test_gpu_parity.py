"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: interaction points within 1e-4 m, path lengths within 1e-6
relative, validity masks identical except for points within 1e-5 m of a
boundary (oracle boundary distance), enumeration bit-exact.  A path is
compared where the oracle reaches a regular minimiser (converged, not
degenerate or repeated) and the GPU reports it solved; the share of such
oracle paths that the GPU fails to solve is bounded separately.
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu

X_TOL = 1e-4
L_RTOL = 1e-6
MASK_MARGIN = 1e-5


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


def to_np(out):
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def gpu_run(ctx, sc, lo, hi, params=None, backward=None):
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, lo, hi, sc.alphabet)
    out = fpt.solve(ctx, scene, batch, params)
    ctx.sync()
    return scene, batch, out


def regular(st):
    return ((st & oracle.CONVERGED) > 0) & ((st & (oracle.DEGENERATE | oracle.REPEAT | oracle.NONFINITE)) == 0)


def min_segments(sc, ids, order, ti, ri, X):
    out = np.full(len(order), np.inf)
    for p in range(len(order)):
        n = order[p]
        pts = np.vstack([sc.tx[ti[p]], X[p, :n], sc.rx[ri[p]]])
        out[p] = np.linalg.norm(np.diff(pts, axis=0), axis=1).min()
    return out


def oracle_solve(sc, ids, order, ti, ri, **kw):
    ref = oracle.solve(sc, ids, order, ti, ri, **kw)
    ref["minseg"] = min_segments(sc, ids, order, ti, ri, ref["X"])
    return ref


def check_parity(g, ref, min_solved_frac=0.99):
    gst, ost = g["status"].astype(np.int32), ref["status"]
    # bit-exact flags decided by integers
    assert np.array_equal((gst & fpt.ST_REPEAT) > 0, (ost & oracle.REPEAT) > 0)
    reg = regular(ost)
    solved = (gst & fpt.ST_SOLVED) > 0
    both = reg & solved
    frac = both.sum() / max(1, reg.sum())
    assert frac >= min_solved_frac, f"GPU solved {frac:.4f} of the oracle's regular paths"
    n = ref["X"].shape[1]
    dx = np.linalg.norm(g["X"][both] - ref["X"][both], axis=2)
    # unused slots are zero on both sides
    assert np.nanmax(dx) <= X_TOL, np.nanmax(dx)
    rel = np.abs(g["L"][both] - ref["L"][both]) / ref["L"][both]
    assert rel.max() <= L_RTOL, rel.max()
    far = both & (np.abs(ref["bdist"]) > MASK_MARGIN)
    assert np.array_equal((gst[far] & fpt.ST_VALID) > 0, (ost[far] & oracle.VALID) > 0)
    # a GPU-solved path is never one whose exact minimiser is a kink (clear of the 1 mm threshold)
    kink = ((ost & oracle.DEGENERATE) > 0) & (ref["minseg"] < 0.5e-3)
    assert not np.any(solved & kink), "solved a degenerate path"
    # every solved path has its residual below the bound, every reported residual is finite when solved
    assert np.all(g["rho"][solved] <= 1e-5)
    return both, n


# ---------------------------------------------------------------------------
# enumeration (bit-exact)
# ---------------------------------------------------------------------------
def test_enumeration_exhaustive_bit_exact(ctx):
    sc = scenes.tiny_scene(0, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 3)
    ids, order, ti, ri = (t.cpu().numpy() for t in fpt.enumerate(ctx, batch))
    e_ids, e_order, e_ti, e_ri = oracle.exhaustive_paths(sc, 1, 3)
    assert np.array_equal(order, e_order) and np.array_equal(ti, e_ti) and np.array_equal(ri, e_ri)
    assert np.array_equal(ids, e_ids)


def test_enumeration_alphabet_and_seeded_bit_exact(ctx):
    sc = scenes.urban_canyon(0, rx_grid=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    ids, order, ti, ri = (t.cpu().numpy() for t in fpt.enumerate(ctx, batch))
    g = np.random.default_rng(0).choice(len(order), 3000, replace=False)
    e = oracle.exhaustive_paths(sc, 3, 3, g)
    assert np.array_equal(ids[g], e[0]) and np.array_equal(ri[g], e[3])
    sb = fpt.Batch.seeded(ctx, scene, 987654321, 5000, 1, 5, sc.alphabet)
    ids, order, ti, ri = (t.cpu().numpy() for t in fpt.enumerate(ctx, sb))
    e = oracle.seeded_paths(sc, 987654321, 5000, 1, 5)
    assert np.array_equal(order, e[1]) and np.array_equal(ids, e[0]) and np.array_equal(ri, e[3])


# ---------------------------------------------------------------------------
# forward parity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(10))
def test_tiny_scene_parity(ctx, seed):
    """10 m box, 8 rectangles + 4 edges, orders 1-2 (156 paths) + order 3 (1728)."""
    sc = scenes.tiny_scene(seed)
    _, _, out = gpu_run(ctx, sc, 1, 3)
    g = to_np(out)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
    ref = oracle_solve(sc, ids, order, ti, ri)
    check_parity(g, ref)


@pytest.mark.parametrize("params", [{}, {"max_iters": 32, "kink_stop": 0.01}], ids=["defaults", "bench"])
def test_urban_canyon_full_size_sampled(ctx, params):
    """33,554,432 order-3 paths on the GPU; 4000 sampled paths re-solved by the oracle (library defaults, and the
    step cap and kink stop the benchmark runs with)."""
    sc = scenes.urban_canyon(0)
    _, batch, out = gpu_run(ctx, sc, 3, 3, fpt.default_params(**params))
    assert batch.n_paths == 32 ** 3 * 1024
    rng = np.random.default_rng(7)
    gidx = np.sort(rng.choice(batch.n_paths, 4000, replace=False))
    import torch

    gi = torch.as_tensor(gidx, device=out["T"].device)
    g = {k: v[gi].cpu().numpy() for k, v in out.items() if v is not None}
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 3, 3, gidx)
    ref = oracle_solve(sc, ids, order, ti, ri)
    check_parity(g, ref, min_solved_frac=0.995)
    # properties over every path
    st = out["status"]
    solved = (st & fpt.ST_SOLVED) > 0
    assert bool((out["rho"][solved] <= 1e-5).all())
    assert not bool(((st & fpt.ST_REPEAT) > 0)[solved].any())
    n_rep = int(((st & fpt.ST_REPEAT) > 0).sum())
    assert n_rep == 1024 * (32 ** 3 - 32 * 31 * 31)  # sequences with an immediate repeat


def test_seeded_city_orders_1_to_5(ctx):
    """Ragged orders 1-5 on a city scene through the order buckets (seeded sequences)."""
    sc = scenes.city(0, n_rx=4)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 42, 1500, 1, 5)
    out = fpt.solve(ctx, scene, batch)
    ctx.sync()
    g = to_np(out)
    ids, order, ti, ri = oracle.seeded_paths(sc, 42, 1500, 1, 5)
    ref = oracle_solve(sc, ids, order, ti, ri)
    check_parity(g, ref, min_solved_frac=0.99)


def test_lane_refill_is_bit_identical(ctx):
    """A path's arithmetic does not depend on which lane runs it: refill on/off give identical bits."""
    sc = scenes.city(1, n_rx=3)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 5, 4000, 1, 5)
    a = to_np(fpt.solve(ctx, scene, batch, fpt.default_params(refill=0)))
    b = to_np(fpt.solve(ctx, scene, batch, fpt.default_params(refill=8)))
    c = to_np(fpt.solve(ctx, scene, batch, fpt.default_params(refill=32)))
    ctx.sync()
    for k in ("T", "status", "iters", "L"):
        assert np.array_equal(a[k], b[k], equal_nan=True) and np.array_equal(a[k], c[k], equal_nan=True), k


def _bits(ctx, scene, batch, **kw):
    out = to_np(fpt.solve(ctx, scene, batch, fpt.default_params(**kw)))
    ctx.sync()
    return out


@pytest.mark.parametrize("case", ["canyon", "city", "tiny_quads_only", "tiny_edges_only"])
def test_pattern_kernels_match_unified_kernel(ctx, case):
    """The interaction-type pattern kernels drop the edges' always-zero second parameter; iterates,
    iteration counts, lengths and flags are bit-identical to the unified d = 2 kernel."""
    if case == "canyon":
        sc = scenes.urban_canyon(0, rx_grid=4)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    elif case == "city":
        sc = scenes.city(2, n_rx=3)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.seeded(ctx, scene, 9, 6000, 1, 5)
    else:
        quads = case == "tiny_quads_only"
        sc = scenes.tiny_scene(3, n_quads=6 if quads else 0, n_edges=0 if quads else 6, n_rx=2)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.exhaustive(ctx, scene, 1, 3, sc.alphabet)
    a = _bits(ctx, scene, batch, specialize=0)
    b = _bits(ctx, scene, batch, specialize=2)  # pattern kernels for every order, however small the buckets
    for k in ("T", "status", "iters", "L", "X", "rho"):
        if a.get(k) is not None:
            assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_batch_refuses_scene_with_other_types(ctx):
    sc = scenes.tiny_scene(1)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 2)
    types = sc.types.copy()
    k = int(np.argmax(types == scenes.QUAD))
    types[k] = scenes.EDGE
    verts = sc.verts.copy()
    verts[k, 2] = 0.0
    other = fpt.Scene(ctx, types, verts, sc.tx, sc.rx)
    with pytest.raises(fpt.FptError):
        fpt.solve(ctx, other, batch)
    ctx.sync()


@pytest.mark.parametrize("seed", [0, 5])
def test_fp64_polish_parity(ctx, seed):
    """The FP64 polish (validation mode) meets the same bars as the double-float default."""
    sc = scenes.tiny_scene(seed)
    _, _, out = gpu_run(ctx, sc, 1, 3, fpt.default_params(polish_fp64=1))
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
    check_parity(to_np(out), oracle_solve(sc, ids, order, ti, ri))


def test_validity_and_residual_at_given_parameters(ctx):
    """fpt_validity at oracle solutions shifted by a seeded perturbation."""
    import torch

    sc = scenes.tiny_scene(3)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    ref = oracle.solve(sc, ids, order, ti, ri)
    rng = np.random.default_rng(5)
    T = ref["T"] + rng.standard_normal(ref["T"].shape) * 2e-5
    T[:, :, 1] = np.where(sc.types[np.maximum(ids, 0)] == scenes.EDGE, 0.5, T[:, :, 1])
    T = T.astype(np.float32)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 2)
    mask, bd, rho = (t.cpu().numpy() for t in fpt.validity(ctx, scene, batch, torch.as_tensor(T, device="cuda")))
    ctx.sync()
    reg = regular(ref["status"])
    for p in np.nonzero(reg)[0]:
        path = oracle.path_from_scene(sc, ids[p, :order[p]], ti[p], ri[p])
        t64 = T[p, :order[p]].astype(np.float64)
        r_ref = path.residual(t64)
        assert abs(rho[p] - r_ref) <= 1e-3 * r_ref + 2e-6, (p, rho[p], r_ref)
        inside = all((0 <= t64[i, 0] <= 1) and (sc.types[ids[p, i]] == scenes.EDGE or 0 <= t64[i, 1] <= 1)
                     for i in range(order[p]))
        assert bool(mask[p]) == inside


# ---------------------------------------------------------------------------
# backward parity (implicit differentiation)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(4))
def test_backward_parity_tiny(ctx, seed):
    """Gradients of sum_i w_i . x_i* + sum valid L* w.r.t. TX, RX and every vertex vs the oracle VJP.

    The oracle's per-path VJPs use weights decided by the oracle alone (regular
    paths away from kinks); the comparison sums them over the paths the GPU also
    solved, and the GPU gets the same weights on those paths.
    """
    import torch

    sc = scenes.tiny_scene(seed, n_rx=2)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    ref = oracle_solve(sc, ids, order, ti, ri)
    st = ref["status"]
    keep = regular(st) & (ref["minseg"] > 0.01)
    dX, dL = scenes.cotangents(100 + seed, len(order), 2)
    dX = dX * keep[:, None, None]
    dL = np.where((st & oracle.VALID) > 0, 1.0, 0.3 * dL) * keep
    ref = oracle.solve(sc, ids, order, ti, ri, dX=dX, dL=dL)
    scene, batch, out = gpu_run(ctx, sc, 1, 2)
    gsolved = (out["status"].cpu().numpy() & fpt.ST_SOLVED) > 0
    both = keep & gsolved
    assert both.sum() >= 0.98 * keep.sum()
    e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, ref["dtheta"] * both[:, None])
    dev = out["T"].device
    w = both.astype(np.float64)
    g_tx, g_rx, g_v = fpt.backward(ctx, scene, batch, out["T"], None,
                                   torch.as_tensor(dX * w[:, None, None], dtype=torch.float32, device=dev),
                                   torch.as_tensor(dL * w, dtype=torch.float32, device=dev))
    ctx.sync()
    scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), 1.0)
    np.testing.assert_allclose(g_tx.cpu().numpy(), e_tx, atol=2e-4 * scale)
    np.testing.assert_allclose(g_rx.cpu().numpy(), e_rx, atol=2e-4 * scale)
    np.testing.assert_allclose(g_v.cpu().numpy(), e_v, atol=2e-4 * scale)


def test_backward_per_path_parity(ctx):
    """Each path's gradient alone (one-hot cotangents) against the oracle's per-path VJP."""
    import torch

    sc = scenes.tiny_scene(0, n_rx=2)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    ref = oracle_solve(sc, ids, order, ti, ri)
    keep = regular(ref["status"]) & (ref["minseg"] > 0.01)
    dX, dL = scenes.cotangents(7, len(order), 2)
    ref = oracle.solve(sc, ids, order, ti, ri, dX=dX * keep[:, None, None], dL=dL * keep)
    scene, batch, out = gpu_run(ctx, sc, 1, 2)
    gsolved = (out["status"].cpu().numpy() & fpt.ST_SOLVED) > 0
    dev = out["T"].device
    worst = 0.0
    for p in np.nonzero(keep & gsolved)[0]:
        one = np.zeros(len(order))
        one[p] = 1.0
        e_tx, e_rx, e_v = oracle.reduce_gradients(sc, ids, order, ti, ri, ref["dtheta"] * one[:, None])
        g_tx, g_rx, g_v = fpt.backward(ctx, scene, batch, out["T"], None,
                                       torch.as_tensor(dX * one[:, None, None], dtype=torch.float32, device=dev),
                                       torch.as_tensor(dL * one, dtype=torch.float32, device=dev))
        scale = max(np.abs(e_v).max(), np.abs(e_tx).max(), np.abs(e_rx).max(), 1.0)
        err = max(np.abs(g_tx.cpu().numpy() - e_tx).max(), np.abs(g_rx.cpu().numpy() - e_rx).max(),
                  np.abs(g_v.cpu().numpy() - e_v).max()) / scale
        worst = max(worst, err)
        assert err < 2e-4, (p, ids[p], err)
    assert worst >= 0.0


def test_backward_valid_length_mask(ctx):
    """dL from the status mask equals an explicit dL = mask."""
    import torch

    sc = scenes.tiny_scene(1)
    scene, batch, out = gpu_run(ctx, sc, 1, 2)
    m = fpt.ST_VALID | fpt.ST_SOLVED
    a = fpt.backward(ctx, scene, batch, out["T"], out["status"], None, None, dL_status_mask=m)
    dL = ((out["status"] & m) == m).float()
    b = fpt.backward(ctx, scene, batch, out["T"], out["status"], None, dL)
    ctx.sync()
    for x, y in zip(a, b):
        torch.testing.assert_close(x, y, rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_zero_iterations_and_fixed_count(ctx):
    sc = scenes.tiny_scene(2)
    _, _, out = gpu_run(ctx, sc, 1, 2, fpt.default_params(max_iters=0))
    g = to_np(out)
    assert not np.any(g["status"] & fpt.ST_CONVERGED)
    assert np.all(g["iters"] == 0)
    _, _, out = gpu_run(ctx, sc, 1, 2, fpt.default_params(max_iters=16, fixed_iters=1))
    g = to_np(out)
    run = (g["status"] & (fpt.ST_REPEAT | fpt.ST_INVALID_INPUT)) == 0
    early = (g["status"] & fpt.ST_NONFINITE) > 0
    assert np.all(g["iters"][run & ~early] <= 16)


def test_explicit_batch_with_invalid_entries(ctx):
    import torch

    sc = scenes.tiny_scene(4)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    ids = torch.tensor([[0, 5, -1], [3, 3, 0], [1, 99, 2], [7, 8, 9], [2, 0, 0]], dtype=torch.int32, device="cuda")
    order = torch.tensor([2, 2, 3, 7, 1], dtype=torch.uint8, device="cuda")
    txi = torch.zeros(5, dtype=torch.int32, device="cuda")
    rxi = torch.tensor([0, 0, 0, 0, 4], dtype=torch.int32, device="cuda")
    batch = fpt.Batch.explicit(ctx, scene, ids, order, txi, rxi)
    out = fpt.solve(ctx, scene, batch)
    ctx.sync()
    st = out["status"].cpu().numpy()
    assert not (st[0] & fpt.ST_INVALID_INPUT)
    assert st[1] & fpt.ST_REPEAT
    assert st[2] & fpt.ST_INVALID_INPUT and st[3] & fpt.ST_INVALID_INPUT and st[4] & fpt.ST_INVALID_INPUT
    e = oracle.solve(sc, np.array([[0, 5]]), np.array([2]), np.array([0]), np.array([0]))
    if regular(e["status"])[0] and st[0] & fpt.ST_SOLVED:
        assert np.linalg.norm(out["X"].cpu().numpy()[0, :2] - e["X"][0]) < X_TOL


def test_ragged_small_batches(ctx):
    """Batches that are not a multiple of a warp, and a single-object scene."""
    sc = scenes.tiny_scene(6, n_quads=1, n_edges=0)
    _, batch, out = gpu_run(ctx, sc, 1, 1)
    assert batch.n_paths == 1
    g = to_np(out)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 1)
    ref = oracle.solve(sc, ids, order, ti, ri)
    if regular(ref["status"])[0]:
        assert g["status"][0] & fpt.ST_SOLVED
        assert np.linalg.norm(g["X"][0, 0] - ref["X"][0, 0]) < X_TOL
    sc = scenes.tiny_scene(6, n_quads=3, n_edges=2, n_rx=3)
    _, batch, out = gpu_run(ctx, sc, 1, 2)
    assert batch.n_paths == 3 * 30
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    check_parity(to_np(out), oracle_solve(sc, ids, order, ti, ri), min_solved_frac=0.98)


def test_bad_arguments_are_errors_not_faults(ctx):
    sc = scenes.tiny_scene(0)
    with pytest.raises(fpt.FptError):
        fpt.Scene(ctx, sc.types, np.full_like(sc.verts, np.nan))
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    with pytest.raises(fpt.FptError):
        fpt.Batch.exhaustive(ctx, scene, 0, 2)
    with pytest.raises(fpt.FptError):
        fpt.Batch.exhaustive(ctx, scene, 1, 11)
    with pytest.raises(fpt.FptError):
        fpt.Batch.exhaustive(ctx, scene, 1, 2, alphabet=[0, 99])
    flat = sc.verts.copy()
    flat[0, 1] = flat[0, 0]
    flat[0, 2] = flat[0, 0]
    with pytest.raises(fpt.FptError):
        fpt.Scene(ctx, sc.types, flat)
    ctx.sync()


def test_fixed_point_rounds_reach_the_oracle_in_fewer_steps(ctx):
    """Sec. IV-A: more Eq. 6 rounds per step converge in fewer steps (fixed step counts, no polish), and the
    reduced d = 1 kernels for diffractions give exactly the unified d = 2 iterates."""
    sc = scenes.tiny_scene(3, n_quads=0, n_edges=12)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 103, 1000, 3, 3)
    ids, order, ti, ri = oracle.seeded_paths(sc, 103, 1000, 3, 3)
    ref = oracle_solve(sc, ids, order, ti, ri)
    keep = regular(ref["status"])
    assert keep.sum() > 500

    def err(k, fp, spec):
        out = to_np(fpt.solve(ctx, scene, batch, fpt.default_params(max_iters=k, fixed_iters=1, fp_iters=fp,
                                                                     polish=0, specialize=spec)))
        ctx.sync()
        e = np.linalg.norm(out["X"][keep] - ref["X"][keep], axis=2).mean(axis=1)
        return e[np.isfinite(e)].mean(), out

    e1, o1 = err(8, 1, 2)
    e64, _ = err(8, 64, 2)
    assert e64 < 0.5 * e1, (e1, e64)
    _, o_unified = err(8, 1, 0)
    assert np.array_equal(o1["T"], o_unified["T"])
    e_late, _ = err(32, 1, 2)
    assert e_late < 1e-5


def test_empty_explicit_batch(ctx):
    """A batch of zero paths: every call succeeds, writes nothing per path and returns zero gradients."""
    import torch

    sc = scenes.tiny_scene(2, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    dev = torch.device("cuda", 0)
    batch = fpt.Batch.explicit(ctx, scene, torch.empty((0, 3), dtype=torch.int32, device=dev),
                               torch.empty(0, dtype=torch.uint8, device=dev), torch.empty(0, dtype=torch.int32, device=dev),
                               torch.empty(0, dtype=torch.int32, device=dev))
    assert batch.n_paths == 0
    out = fpt.solve(ctx, scene, batch)
    assert out["T"].shape == (0, 3, 2) and out["status"].shape == (0,)
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    out, (g_tx, g_rx, g_v) = fpt.solve_grad(ctx, scene, batch, dL_status_mask=mask)
    ctx.sync()
    assert fpt.count_status(ctx, out["status"], mask) == 0
    for g in (g_tx, g_rx, g_v):
        assert g.numel() > 0 and not g.any()
    g_tx, g_rx, g_v = fpt.backward(ctx, scene, batch, out["T"], out["status"], dL_status_mask=mask)
    ctx.sync()
    assert not (g_tx.any() or g_rx.any() or g_v.any())
    m, bd, rho = fpt.validity(ctx, scene, batch, out["T"])
    assert m.numel() == 0
    assert fpt.occlusion(ctx, scene, batch, out["T"], out["status"], mask).numel() == 0
    ids, order, ti, ri = fpt.enumerate(ctx, batch)
    ctx.sync()
    assert ids.shape == (0, 3) and order.numel() == 0


def test_degenerate_geometries_are_never_solved(ctx):
    """Endpoints on an object, on an edge's line and at the same point: the minimisers with a
    zero-length segment (kinks of L, DEGENERATE in the oracle) are never reported SOLVED, nothing
    turns non-finite, and the regular cases still meet the oracle."""
    quad = np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 0.0], [0.0, 10.0, 0.0]])  # the plane z = 0
    edge = np.array([[0.0, 12.0, 0.0], [0.0, 12.0, 10.0], [0.0, 0.0, 0.0]])  # the line x = 0, y = 12
    types = np.array([scenes.QUAD, scenes.EDGE], dtype=np.uint8)
    verts = np.stack([quad, edge])
    tx = np.array([[5.0, 5.0, 0.0],       # on the plane
                   [0.0, 12.0, 4.0],      # on the edge
                   [3.0, 4.0, 2.0]])      # regular
    rx = np.array([[5.0, 5.0, 3.0], [3.0, 4.0, 2.0]])  # the second RX coincides with the third TX
    sc = scenes.Scene(types, verts, tx, rx)
    _, batch, out = gpu_run(ctx, sc, 1, 2)
    g = to_np(out)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 2)
    ref = oracle_solve(sc, ids, order, ti, ri)
    gst, ost = g["status"].astype(np.int32), ref["status"]
    assert not (gst & fpt.ST_NONFINITE).any()
    deg = (ost & oracle.DEGENERATE) > 0
    assert deg.sum() >= 3
    assert not ((gst & fpt.ST_SOLVED) > 0)[deg].any()
    assert regular(ost).sum() >= 8
    check_parity(g, ref, min_solved_frac=0.9)


def test_largest_scene_uses_the_full_16_bit_object_ids(ctx):
    """65,535 objects (the most a scene holds: bucket records keep 16-bit ids): seeded sequences
    over all of them meet the oracle; one object more is an argument error."""
    rng = np.random.default_rng(17)
    K = 65535
    types = (rng.random(K) < 0.3).astype(np.uint8)  # ~30 % edges
    verts = np.zeros((K, 3, 3))
    for k in range(K):
        verts[k] = scenes.random_edge(rng, 1, 3, 1, 9) if types[k] else scenes.random_rectangle(rng, 1, 4, 1, 9)
    tx = rng.uniform(0, 10, (1, 3))
    rx = rng.uniform(0, 10, (2, 3))
    sc = scenes.Scene(types, verts, tx, rx)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 5, 1500, 1, 3)
    out = to_np(fpt.solve(ctx, scene, batch))
    ctx.sync()
    ids, order, ti, ri = oracle.seeded_paths(sc, 5, 1500, 1, 3)
    assert ids.max() > 60000
    check_parity(out, oracle_solve(sc, ids, order, ti, ri), min_solved_frac=0.98)
    with pytest.raises(fpt.FptError):
        fpt.Scene(ctx, np.zeros(K + 1, dtype=np.uint8), np.concatenate([verts, verts[:1]]))
