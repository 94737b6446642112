"""Warm-start network on the tensor cores against the FP64 reference (GPU)."""

import os

import numpy as np
import pytest

import oracle
from oracle import mlp_oracle as mo
from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu
SCALE = 10.0


@pytest.fixture(scope="module")
def ctx():
    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    return fpt.Context(0)


def numpy_params(seed):
    rng = np.random.default_rng(seed)
    P = {}
    for name, shape in mo.SIZES:
        if len(shape) == 2:
            P[name] = rng.uniform(-1, 1, shape) / np.sqrt(shape[1])
        else:
            P[name] = 0.05 * rng.standard_normal(shape)
    P["W4"][8:] = 0.0
    P["b4"][8:] = 0.0
    return mo.pack(P).astype(np.float32)


def tiny_batch(ctx, seed, lo=1, hi=3):
    sc = scenes.tiny_scene(seed)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.exhaustive(ctx, scene, lo, hi)
    return sc, scene, batch


def test_features_match_definition(ctx):
    import torch

    sc, scene, batch = tiny_batch(ctx, 0)
    net = fpt.Mlp(ctx, 1, SCALE)
    X, G = net.features(scene, batch, with_gram=True)
    X, G = X.float().cpu().numpy(), G.cpu().numpy()
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
    F, Go = mo.features(sc, ids, order, ti, ri, SCALE)
    F = mo.bf16(F)
    # FP32 projections rounded to bf16 may land one bf16 step away from the FP64 ones
    ulp = np.abs(F) * 2.0 ** -7 + 1e-6
    assert np.all(np.abs(X - F) <= ulp), np.abs(X - F).max()
    np.testing.assert_allclose(G, Go, rtol=1e-5, atol=1e-7)
    assert torch.cuda.is_available()


def test_forward_and_gradient_match_reference(ctx):
    import torch

    sc, scene, batch = tiny_batch(ctx, 1)
    params = numpy_params(5)
    net = fpt.Mlp(ctx, 0, SCALE)
    net.set_params(params)
    X, G = net.features(scene, batch, with_gram=True)
    ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
    Fo, Go = mo.features(sc, ids, order, ti, ri, SCALE)
    Xo = mo.bf16(Fo)
    Y = net.forward(X).cpu().numpy()
    Yo = mo.forward(params.astype(np.float64), Xo)["Y"]
    assert np.abs(Y - Yo).max() <= 5e-3 * max(1.0, np.abs(Yo).max())
    T = np.random.default_rng(6).uniform(-0.5, 1.5, (len(order), 8))
    loss, g = net.loss_grad(X, torch.as_tensor(T, dtype=torch.float32, device="cuda"), G)
    lo, go = mo.loss_grad(params.astype(np.float64), Xo, T, Go)
    assert abs(loss - lo) <= 2e-3 * abs(lo)
    g = g.cpu().numpy()
    assert np.abs(g - go).max() <= 3e-3 * np.abs(go).max(), (np.abs(g - go).max(), np.abs(go).max())
    # the padded outputs stay zero
    assert np.all(g[mo.N_PARAMS - 16 - 8 * 256 - 8:mo.N_PARAMS - 16] == 0)


@pytest.mark.parametrize("n", [4096, 40001, 40008])
def test_gradient_at_a_large_ragged_batch(ctx, n):
    """Random samples: at 40,001 and 40,008 rows 313 row tiles (the last one ragged), so every CTA of the
    persistent GEMM runs two or three tiles through both TMEM accumulators and wraps its operand ring; the
    weight gradients split K (the batch) over 126 slices.  4096 and 40,008 rows give transposed
    activations whose row stride a tensor map can describe (TMA tensor stores); 40,001 rows do not (the
    lanes store them).  Forward, loss and gradient against the FP64 reference with the same BF16
    roundings."""
    import torch

    rng = np.random.default_rng(11)
    Xo = mo.bf16(rng.uniform(-1.0, 1.0, (n, 64)))
    G = rng.normal(0.0, 1.0, (n, 4, 3))
    T = rng.uniform(-0.5, 1.5, (n, 8))
    params = numpy_params(7)
    net = fpt.Mlp(ctx, 0, SCALE)
    net.set_params(params)
    X = torch.as_tensor(Xo, dtype=torch.float32).to(torch.bfloat16).cuda()
    Y = net.forward(X).cpu().numpy()
    Yo = mo.forward(params.astype(np.float64), Xo)["Y"]
    assert np.abs(Y - Yo).max() <= 5e-3 * max(1.0, np.abs(Yo).max())
    loss, g = net.loss_grad(X, torch.as_tensor(T, dtype=torch.float32, device="cuda"),
                            torch.as_tensor(G, dtype=torch.float32, device="cuda"))
    lo, go = mo.loss_grad(params.astype(np.float64), Xo, T, G)
    assert abs(loss - lo) <= 2e-3 * abs(lo)
    g = g.cpu().numpy()
    assert np.abs(g - go).max() <= 3e-3 * np.abs(go).max(), (np.abs(g - go).max(), np.abs(go).max())


def training_set(ctx, seeds, per_pair=20000):
    """Features and solver outputs (solved paths only) for seeded order 1-4 sequences on tiny scenes."""
    import torch

    from paper_2510_16172_gb300 import warmstart

    return warmstart.make_dataset(ctx, seeds, per_pair)


def test_training_reduces_loss_and_checkpoint_resumes(ctx, tmp_path):
    X, T, G = training_set(ctx, [11, 12, 13])
    net = fpt.Mlp(ctx, 3, SCALE)
    B = 4096
    n = X.shape[0] // B * B
    first = net.loss_grad(X[:n], T[:n], G[:n])[0]
    for step in range(200):
        k = (step * B) % n
        net.train_step(X[k:k + B], T[k:k + B], G[k:k + B], 2e-3, want_loss=False)
    path = os.path.join(tmp_path, "net.bin")
    net.save(path)
    mid = net.loss_grad(X[:n], T[:n], G[:n])[0]
    assert mid < 0.6 * first, (first, mid)
    other = fpt.Mlp.load(ctx, path)
    np.testing.assert_array_equal(other.get_params(), net.get_params())
    for step in range(200, 220):
        k = (step * B) % n
        la = net.train_step(X[k:k + B], T[k:k + B], G[k:k + B], 1e-3)
        lb = other.train_step(X[k:k + B], T[k:k + B], G[k:k + B], 1e-3)
        assert abs(la - lb) <= 1e-3 * abs(la)


def test_learned_start_keeps_parity(ctx):
    from test_gpu_parity import check_parity, oracle_solve, to_np

    X, T, G = training_set(ctx, [21, 22])
    net = fpt.Mlp(ctx, 4, SCALE)
    B = 4096
    n = X.shape[0] // B * B
    for step in range(100):
        k = (step * B) % n
        net.train_step(X[k:k + B], T[k:k + B], G[k:k + B], 1e-3, want_loss=False)
    net.attach()
    for seed in (31, 32):
        sc, scene, batch = tiny_batch(ctx, seed)
        out = fpt.solve(ctx, scene, batch, fpt.default_params(init_mode=1))
        ctx.sync()
        ids, order, ti, ri = oracle.exhaustive_paths(sc, 1, 3)
        # From this network's start BFGS ends 0.7-1.1 % of seed 32's 1016 regular paths elsewhere (a kink
        # stop or the step cap) over seven trainings on the GB300, against 0.3 % from the plain start.
        # Training is not bit-reproducible (float atomics in its gradient sums), so the bound leaves room
        # for that spread: at least 98.5 % solved, at the usual tolerances.
        check_parity(to_np(out), oracle_solve(sc, ids, order, ti, ri), min_solved_frac=0.985)


@pytest.mark.parametrize("seed,kind,lo,hi", [(41, "seeded", 1, 5), (42, "seeded", 1, 5), (43, "exhaustive", 1, 3),
                                              (44, "seeded", 6, 8)])
def test_fused_inference_start_matches_reference(ctx, seed, kind, lo, hi):
    """The fused tensor-core inference writes the network's prediction as the start (checked with no BFGS
    steps), for each path source: bucket records of orders 1-5 (9000 paths, ragged last tile), an
    exhaustive batch's enumeration, and records of orders 6-8 (ids decoded again; slots 5+ start at 1/2)."""
    params = numpy_params(seed)
    net = fpt.Mlp(ctx, 0, SCALE)
    net.set_params(params)
    net.attach()
    sc = scenes.tiny_scene(seed, n_rx=3)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    if kind == "seeded":
        batch = fpt.Batch.seeded(ctx, scene, seed, 3000, lo, hi)
        ids, order, ti, ri = oracle.seeded_paths(sc, seed, 3000, lo, hi)
    else:
        batch = fpt.Batch.exhaustive(ctx, scene, lo, hi)
        ids, order, ti, ri = oracle.exhaustive_paths(sc, lo, hi)
    out = fpt.solve(ctx, scene, batch, fpt.default_params(init_mode=1, max_iters=0, polish=0))
    ctx.sync()
    T = out["T"].cpu().numpy()
    keep = (out["status"].cpu().numpy() & fpt.ST_REPEAT) == 0  # repeats are not solved
    assert keep.sum() > 1000
    Fo, _ = mo.features(sc, ids, order, ti, ri, SCALE)
    Y = mo.forward(params.astype(np.float64), mo.bf16(Fo))["Y"]
    expect = np.full(T.shape, 0.5)
    for p in range(len(order)):
        for s in range(min(order[p], 4)):
            expect[p, s, 0] = Y[p, 2 * s]
            if sc.types[ids[p, s]] == scenes.QUAD:
                expect[p, s, 1] = Y[p, 2 * s + 1]
    used = (np.arange(T.shape[1])[None, :] < order[:, None]) & keep[:, None]
    err = np.abs(T - expect)[used]
    assert err.max() <= 5e-3 * max(1.0, np.abs(Y).max()), err.max()


def test_mlp_infer_is_the_solver_start(ctx):
    """fpt_mlp_infer writes the learned start the solver begins from: a solve with no BFGS steps and no
    polish returns exactly it (seeded orders 1-5, a ragged batch, unused slots zero)."""
    import torch

    sc = scenes.city(1, n_rx=2)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 3, 5000, 1, 5)
    net = fpt.Mlp(ctx, 0, SCALE)
    net.set_params(numpy_params(4))
    start = net.infer(scene, batch)
    net.attach()
    out = fpt.solve(ctx, scene, batch, fpt.default_params(init_mode=1, max_iters=0, polish=0))
    ctx.sync()
    assert torch.equal(start, out["T"])
    _, order, _, _ = fpt.enumerate(ctx, batch)
    unused = torch.arange(batch.n_max, device=order.device)[None, :] >= order.long()[:, None]
    assert bool((start[unused] == 0).all())
    net.close()


def test_mlp_train_native_schedule(ctx):
    """fpt_mlp_train: the epoch loop in the library lowers the loss, and the seed fixes the sample order
    (the same seed reproduces a run up to the rounding order of atomic sums, another seed does not)."""
    from paper_2510_16172_gb300 import warmstart

    X, T, G = warmstart.make_dataset(ctx, [31, 32], 20000)
    runs = []
    for seed in (5, 5, 6):
        net = fpt.Mlp(ctx, 2, SCALE)
        hist = net.train(X, T, G, epochs=4, batch=4096, lr=1e-3, lr_decay=0.7, seed=seed)
        runs.append((hist, net.get_params()))
        net.close()
    hist = runs[0][0]
    assert len(hist) == 4 and all(np.isfinite(hist))
    assert hist[-1] < 0.8 * hist[0], hist
    # the same seed gives the same sample order; only the float atomics of the split-K weight-gradient
    # sums differ in rounding order, so two runs agree far more closely than runs with other orders
    same = np.abs(runs[0][1] - runs[1][1]).max()
    other = np.abs(runs[0][1] - runs[2][1]).max()
    assert same < 0.05 * other, (same, other)
    assert abs(runs[0][0][-1] - runs[1][0][-1]) <= 1e-3 * runs[0][0][-1]


def test_mlp_train_full_batch_epoch_is_one_step(ctx):
    """One epoch of fpt_mlp_train with the batch = every sample is one Adam step on a shuffled copy of the
    whole set, so it equals one fpt_mlp_train_step on the unshuffled set up to the summation order.  Adam's
    first step moves each weight by +-lr (sign of its gradient), so the layers agree entry by entry except
    where a gradient is at the rounding level: a wrong shuffle of X, T, G or of the transposed features the
    library gathers for the first layer's weight gradient would flip about half of them."""
    from paper_2510_16172_gb300 import warmstart

    X, T, G = warmstart.make_dataset(ctx, [33, 34], 20000)
    n = min(X.shape[0], 16384) // 8 * 8
    X, T, G = X[:n].contiguous(), T[:n].contiguous(), G[:n].contiguous()
    lr = 1e-3
    a = fpt.Mlp(ctx, 7, SCALE)
    b = fpt.Mlp(ctx, 7, SCALE)
    a.train(X, T, G, epochs=1, batch=n, lr=lr, lr_decay=1.0, seed=3)
    b.train_step(X, T, G, lr, want_loss=False)
    pa, pb = mo.unpack(a.get_params()), mo.unpack(b.get_params())
    for name in ("W1", "b1", "W2", "W3", "W4"):
        flips = np.mean(np.abs(pa[name] - pb[name]) > lr)
        assert flips <= 0.01, (name, flips)
    a.close()
    b.close()


def test_learned_start_saves_steps_on_unseen_scenes(ctx):
    """What the trained network gains (config 4 in small): trained by the library's tensor-core kernels on
    the solver's own solutions of seeded order-1..4 sequences on 20 random 10 m scenes, it starts the solver
    on 5 unseen scenes.  Against the plain start on the same sequences: at least 3 % fewer BFGS steps on
    average, no fewer solved paths than 0.5 % below, and the same stationarity bound on every solved path."""
    import torch

    from paper_2510_16172_gb300 import warmstart

    X, T, G = warmstart.make_dataset(ctx, seeds=tuple(range(1000, 1020)), per_pair=100_000)
    net, hist = warmstart.train(ctx, X, T, G, epochs=6, seed=3)
    del X, T, G
    assert hist[-1] < hist[0]
    ev = warmstart.evaluate(ctx, net, seeds=tuple(range(2000, 2005)), per_pair=100_000, repeats=1)
    net.close()
    plain, learned = ev["plain"], ev["learned"]
    assert learned["mean_bfgs_iters"] <= 0.97 * plain["mean_bfgs_iters"], (learned, plain)
    assert learned["solved"] >= 0.995 * plain["solved"], (learned, plain)
    assert learned["max_rho_solved_m"] <= 1e-5 and plain["max_rho_solved_m"] <= 1e-5
    assert torch.cuda.is_available()
