"""Implicit backward at full size against the oracle (Sec. III-D, Eq. 9-13).

The urban canyon (33,554,432 order-3 paths, the benchmark's settings) and a
10,000,000-path seeded city batch of orders 1-5: the loss is the sum of the
valid solved paths' lengths plus seeded point and length cotangents on 4000
sample paths, differentiated with respect to TX, RX and every vertex.  The
oracle solves every path that carries a cotangent (about 2.2 M on the canyon)
in FP64 and forms its VJP; the GPU sums are compared with the oracle's sums
over the paths that both sides solve (oracle: a regular minimiser with every
segment longer than 1 cm), each gradient array within 2e-4 of its largest
entry.  At these sizes every CTA of the adjoint kernel works through hundreds
of 128-path tiles, so its FP32 shared-memory partial sums are flushed into the
FP64 totals many times; the listed adjoint (length cotangents from a status
mask) runs over about 2.2 M listed paths.  A tiny multi-tile batch also runs
with a flush after every tile, every few tiles and with no shared-memory sums.
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu

REL = 2e-4          # gradient sums: within 2e-4 of the array's largest entry
N_SAMPLES = 4000


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    c = fpt.Context(0)
    yield c
    c.set_accumulation(64, 1)


def regular(st):
    return ((st & oracle.CONVERGED) > 0) & ((st & (oracle.DEGENERATE | oracle.REPEAT | oracle.NONFINITE)) == 0)


def min_segments(sc, order, ti, ri, X):
    """Shortest segment of each path (TX, its points, RX)."""
    M, n_max = X.shape[:2]
    pts = np.concatenate([sc.tx[ti][:, None, :], X, np.zeros((M, 1, 3))], axis=1)
    pts[np.arange(M), order + 1] = sc.rx[ri]
    seg = np.linalg.norm(np.diff(pts, axis=1), axis=2)
    inside = np.arange(n_max + 1)[None, :] <= order[:, None]
    return np.where(inside, seg, np.inf).min(axis=1)


def assert_sums_close(got, want, what, per_array=True):
    """Each gradient array within REL of its own largest entry (per_array), or of the largest entry of
    all three (the bound of the other backward tests)."""
    overall = max(max(np.abs(e).max() for e in want), 1.0)
    for name, g, e in zip(("TX", "RX", "vertices"), got, want):
        g = g.cpu().numpy().astype(np.float64)
        scale = max(np.abs(e).max(), 1.0) if per_array else overall
        err = np.abs(g - e).max()
        assert err <= REL * scale, f"{what}: {name} gradient off by {err:.3e} (scale {scale:.3e})"


# Per-path error of the FP32 adjoint (block LDL^T of the Eq. 12 system, then Eq. 13), measured on the
# GB300 against the oracle's FP64 VJP at the GPU's own parameters, over 20,000 regular tiny-scene paths of
# orders 1-3 with segments above 10 cm: median 2.2e-7, 99th percentile 1.2e-5, largest 3.1e-4 of the
# path's largest gradient entry.  A sum over many paths then differs from the oracle's by at most
# PATH_EPS times the sum of its paths' largest entries, whatever the order of summation.
PATH_EPS = 1e-3


def path_magnitude_bounds(sc, ids, order, tx_idx, rx_idx, dtheta):
    """For every TX, RX and vertex entry, PATH_EPS times the sum over the paths that contribute to it of
    each path's largest |gradient| entry (the vertex chain rule of oracle.reduce_gradients taken with
    absolute values: v0 collects the b, a1 and a2 parameters of its object)."""
    m = np.abs(np.asarray(dtheta, dtype=np.float64)).max(axis=1)
    K = sc.n_obj
    b_tx = np.zeros(len(sc.tx))
    b_rx = np.zeros(len(sc.rx))
    b_obj = np.zeros(K)
    np.add.at(b_tx, np.asarray(tx_idx), m)
    np.add.at(b_rx, np.asarray(rx_idx), m)
    for i in range(ids.shape[1]):
        on = np.asarray(order) > i
        np.add.at(b_obj, np.asarray(ids)[on, i], m[on])
    quad = sc.types == scenes.QUAD
    b_v = np.zeros((K, 3))
    b_v[:, 0] = np.where(quad, 3.0, 2.0) * b_obj
    b_v[:, 1] = b_obj
    b_v[:, 2] = np.where(quad, b_obj, 0.0)
    return (PATH_EPS * b_tx[:, None] + 1e-6, PATH_EPS * b_rx[:, None] + 1e-6, PATH_EPS * b_v[:, :, None] + 1e-6)


def assert_within_path_bounds(got, want, bounds, what):
    for name, g, e, b in zip(("TX", "RX", "vertices"), got, want, bounds):
        g = g.cpu().numpy().astype(np.float64)
        over = np.abs(g - e) / b
        k = np.unravel_index(np.argmax(over), over.shape)
        assert over[k] <= 1.0, f"{what}: {name} gradient {k} off by {abs(g - e)[k]:.3e}, bound {np.broadcast_to(b, g.shape)[k]:.3e}"


def sampled_backward_case(ctx, sc, scene, batch, decode, params, seed):
    """Solve the whole batch on the GPU, then check fpt_backward, its listed form and fpt_solve_grad
    against the oracle's VJP sums (see the module docstring)."""
    import torch

    out = fpt.solve(ctx, scene, batch, params)
    ctx.sync()
    st = out["status"]
    N, n_max = batch.n_paths, batch.n_max
    dev = st.device
    vs_mask = fpt.ST_VALID | fpt.ST_SOLVED
    vs_idx = torch.nonzero((st & vs_mask) == vs_mask).squeeze(1).cpu().numpy()
    rng = np.random.default_rng(seed)
    samp = np.sort(rng.choice(N, N_SAMPLES, replace=False))
    st_h = st.cpu().numpy()

    # oracle: the length cotangent on every GPU-valid solved path ...
    ids_l, order_l, ti_l, ri_l = decode(vs_idx)
    ref_l = oracle.solve(sc, ids_l, order_l, ti_l, ri_l, dL=np.ones(len(vs_idx)))
    keep_l = regular(ref_l["status"]) & (min_segments(sc, order_l, ti_l, ri_l, ref_l["X"]) > 0.01)
    # ... and point and length cotangents on the sample paths
    ids_s, order_s, ti_s, ri_s = decode(samp)
    dXs, dLs = scenes.cotangents(seed, N_SAMPLES, n_max)
    ref_s0 = oracle.solve(sc, ids_s, order_s, ti_s, ri_s)
    keep_s = (regular(ref_s0["status"]) & (min_segments(sc, order_s, ti_s, ri_s, ref_s0["X"]) > 0.01)
              & ((st_h[samp] & fpt.ST_SOLVED) > 0))
    # the GPU solves nearly every path the oracle finds regular
    reg_s = regular(ref_s0["status"]) & (min_segments(sc, order_s, ti_s, ri_s, ref_s0["X"]) > 0.01)
    assert keep_s.sum() >= 0.99 * reg_s.sum(), (keep_s.sum(), reg_s.sum())
    assert keep_l.mean() >= 0.98, keep_l.mean()
    dXs = dXs * keep_s[:, None, None]
    dLs = 0.3 * dLs * keep_s
    ref_s = oracle.solve(sc, ids_s, order_s, ti_s, ri_s, dX=dXs, dL=dLs)
    e_l = oracle.reduce_gradients(sc, ids_l, order_l, ti_l, ri_l, ref_l["dtheta"] * keep_l[:, None])
    e_s = oracle.reduce_gradients(sc, ids_s, order_s, ti_s, ri_s, ref_s["dtheta"])
    e_all = tuple(a + b for a, b in zip(e_l, e_s))

    # GPU cotangent arrays over the whole batch (zero off the chosen paths)
    dX = torch.zeros((N, n_max, 3), dtype=torch.float32, device=dev)
    dL = torch.zeros(N, dtype=torch.float32, device=dev)
    li = torch.as_tensor(vs_idx, device=dev)
    si = torch.as_tensor(samp, device=dev)
    dL[li] = torch.as_tensor(keep_l, dtype=torch.float32, device=dev)
    dL[si] += torch.as_tensor(dLs, dtype=torch.float32, device=dev)
    dX[si] = torch.as_tensor(dXs, dtype=torch.float32, device=dev)

    # 1) point + length cotangents: every path is visited by the adjoint kernel
    got = fpt.backward(ctx, scene, batch, out["T"], st, dX, dL)
    ctx.sync()
    assert_sums_close(got, e_all, "fpt_backward with dX and dL")
    # paths left out as singular even in FP64 are counted (none among regular paths)
    assert 0 <= fpt.backward_dropped(ctx) <= 1e-4 * N

    # 2) length cotangents from the status mask: the listed adjoint over the valid solved paths the
    #    oracle also finds regular (VALID cleared on the others)
    st2 = st.clone()
    drop = torch.as_tensor(vs_idx[~keep_l], device=dev)
    st2[drop] &= ~fpt.ST_VALID
    got = fpt.backward(ctx, scene, batch, out["T"], st2, dL_status_mask=vs_mask)
    ctx.sync()
    assert_sums_close(got, e_l, "fpt_backward with dL_status_mask")

    # 3) the same cotangents given to the fused solve + backward call (both adjoint placements)
    for fuse in (0, 1):
        p = fpt.SolveParams.from_buffer_copy(params)
        p.fuse_adjoint = fuse
        out2, got = fpt.solve_grad(ctx, scene, batch, p, dX=dX, dL=dL)
        ctx.sync()
        if fuse == 0:  # fpt_solve then fpt_backward: the solve's outputs bit for bit
            assert torch.equal(out2["status"], st) and torch.equal(out2["T"], out["T"])
        else:  # the polish instantiation with the adjoint may round a Newton step differently
            assert int((out2["status"] != st).sum()) <= 1e-4 * N
        assert_sums_close(got, e_all, f"fpt_solve_grad (fuse_adjoint={fuse})")
        del out2

    # validity of the returned parameters on the sample paths, solved or not: VALID says that every
    # point lies inside its object at the returned T (closed test), away from rounding at the boundary
    T_s = out["T"][si].cpu().numpy().astype(np.float64)
    quad = sc.types[np.where(ids_s >= 0, ids_s, 0)] == scenes.QUAD
    slot = np.arange(n_max)[None, :] < order_s[:, None]
    t1, t2 = T_s[:, :, 0], T_s[:, :, 1]
    inside_slot = (t1 >= 0) & (t1 <= 1) & (~quad | ((t2 >= 0) & (t2 <= 1)))
    inside = np.where(slot, inside_slot, True).all(axis=1)
    d1 = np.minimum(np.abs(t1), np.abs(t1 - 1))
    d2 = np.where(quad, np.minimum(np.abs(t2), np.abs(t2 - 1)), np.inf)
    clear = np.where(slot, np.minimum(d1, d2), np.inf).min(axis=1) > 1e-5
    run = (st_h[samp] & (fpt.ST_REPEAT | fpt.ST_INVALID_INPUT)) == 0
    chk = run & clear
    assert chk.sum() > 0.9 * run.sum()
    assert np.array_equal((st_h[samp][chk] & fpt.ST_VALID) > 0, inside[chk])
    # sample paths the oracle finds regular but the GPU leaves unsolved: their mask is still the test above
    unsolved = reg_s & ((st_h[samp] & fpt.ST_SOLVED) == 0)
    return int(unsolved.sum())


def test_canyon_full_size_backward_vs_oracle(ctx):
    """33,554,432 paths at the benchmark's settings (step cap 32, kink stop 1 cm)."""
    sc = scenes.urban_canyon(0)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 3, 3, sc.alphabet)
    assert batch.n_paths == 32 ** 3 * 1024
    params = fpt.default_params(max_iters=32, kink_stop=0.01)
    sampled_backward_case(ctx, sc, scene, batch, lambda g: oracle.exhaustive_paths(sc, 3, 3, g), params, 31)


def test_city_10m_backward_vs_oracle(ctx):
    """10,000,000 seeded sequences of order 1-5 on the 256-object city (library defaults)."""
    sc = scenes.city(0, n_rx=16)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    per_pair = 625_000
    batch = fpt.Batch.seeded(ctx, scene, 9, per_pair, 1, 5)
    assert batch.n_paths == 10_000_000
    sampled_backward_case(ctx, sc, scene, batch, lambda g: oracle.seeded_paths(sc, 9, per_pair, 1, 5, g),
                          fpt.default_params(), 32)


def test_backward_sums_by_flush_interval(ctx):
    """241,152 tiny-scene paths (orders 1-3, 128 RX; about three 128-path tiles per CTA of the order-3
    adjoint): fpt_backward, fpt_solve_grad with the fused adjoint and fpt_backward_noalloc with the
    shared-memory partial sums flushed after every tile, every two tiles, every 64 (the default) or not
    used at all.  The reference is the oracle's FP64 VJP (Eq. 12-13) evaluated at the GPU's own solution
    (the oracle's solver run for zero steps from it), so the comparison sees the backward's arithmetic
    and its summation, not the solve's tolerance.  Every setting agrees with it within the per-path FP32
    adjoint error (PATH_EPS of each contributing path's largest entry), and with the sums taken straight
    in FP64 to 1e-5 of the largest entry: the FP32 partial sums add nothing visible to the adjoint's own
    rounding."""
    import torch

    sc = scenes.tiny_scene(3, n_rx=128)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
    ref0 = oracle.solve(sc, ids, order, ti, ri)
    minseg = min_segments(sc, order, ti, ri, ref0["X"])
    keep = regular(ref0["status"]) & (minseg > 0.01)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 3)
    out = fpt.solve(ctx, scene, batch)
    ctx.sync()
    gsolved = (out["status"].cpu().numpy() & fpt.ST_SOLVED) > 0
    assert (keep & gsolved).sum() >= 0.98 * keep.sum()
    # cotangents on paths whose segments are all longer than 10 cm: on centimetre segments the FP32
    # products a t carry ~1e-4 relative error into z, on gradient terms that scale like 1/|z|, which would
    # dominate these sums over 241 k paths without saying anything about the summation under test
    w = keep & gsolved & (minseg > 0.1)
    dX, dL = scenes.cotangents(55, len(order), 3)
    valid = (ref0["status"] & oracle.VALID) > 0
    dL = np.where(valid, 1.0, 0.3 * dL) * w
    dX = dX * w[:, None, None]
    T_gpu = out["T"].cpu().numpy().astype(np.float64)
    ref = oracle.solve(sc, ids, order, ti, ri, solver=oracle.BFGS, max_iters=0, T_start=T_gpu, dX=dX, dL=dL)
    assert np.array_equal(ref["T"][w], T_gpu[w])  # the oracle evaluated at the GPU's parameters
    want = oracle.reduce_gradients(sc, ids, order, ti, ri, ref["dtheta"] * w[:, None])
    bounds = path_magnitude_bounds(sc, ids, order, ti, ri, ref["dtheta"] * w[:, None])
    dev = out["T"].device
    dXd = torch.as_tensor(dX, dtype=torch.float32, device=dev)
    dLd = torch.as_tensor(dL, dtype=torch.float32, device=dev)
    results = {}
    try:
        for flush, smem in ((1, 0), (1, 1), (2, 1), (64, 1)):
            ctx.set_accumulation(flush, smem)
            got = fpt.backward(ctx, scene, batch, out["T"], out["status"], dXd, dLd)
            ctx.sync()
            assert_within_path_bounds(got, want, bounds, f"fpt_backward, flush {flush}, smem {smem}")
            results[(flush, smem)] = [g.cpu().numpy().astype(np.float64) for g in got]
            got = fpt.backward_noalloc(ctx, scene, batch, out["T"], out["status"], dXd, dLd)
            ctx.sync()
            assert_within_path_bounds(got, want, bounds, f"fpt_backward_noalloc, flush {flush}, smem {smem}")
            # the fused adjoint runs at the polish's own (equally solved) point
            _, got = fpt.solve_grad(ctx, scene, batch, fpt.default_params(fuse_adjoint=1), dX=dXd, dL=dLd)
            ctx.sync()
            assert_within_path_bounds(got, want, bounds, f"fpt_solve_grad fused, flush {flush}, smem {smem}")
    finally:
        ctx.set_accumulation(64, 1)
    # FP32 partial sums of up to 64 tiles against sums taken in FP64 path by path
    exact = results[(1, 0)]
    for key, got in results.items():
        for g, e in zip(got, exact):
            assert np.abs(g - e).max() <= 1e-5 * max(np.abs(e).max(), 1.0), key


def test_set_accumulation_rejects_bad_values(ctx):
    with pytest.raises(fpt.FptError):
        ctx.set_accumulation(0, 1)
    with pytest.raises(fpt.FptError):
        ctx.set_accumulation(4, 2)
    ctx.set_accumulation(64, 1)
