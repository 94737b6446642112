"""Learned warm start: training data from the solver itself, training and evaluation.

The network (fpt_mlp_*, tensor-core kernels) learns to predict the solution
parameters of the first four interactions from the sequence geometry.  Its
training set is produced by the solver: seeded batches of order-1..4
sequences on random 10 m scenes are solved, and the solved paths' features
and parameters become (input, target) pairs.  Evaluation solves unseen scenes
twice, from the plain start (t = 1/2) and from the network's prediction, and
compares BFGS iterations, solved paths per second and stationarity.
Everything below is orchestration; all computation runs in libfpt.so.
"""

from __future__ import annotations

import time

from . import fpt, scenes

TRAIN_SEEDS = tuple(range(1000, 1050))
EVAL_SEEDS = tuple(range(2000, 2010))
LENGTH_SCALE = 10.0


def make_dataset(ctx, seeds=TRAIN_SEEDS, per_pair=200_000, order_lo=1, order_hi=4, net=None):
    """Features (bf16 [n, 64]), solved parameters (float [n, 8]) and loss Gram matrices (float [n, 4, 3])
    of the solved paths of seeded batches."""
    import torch

    net = net or fpt.Mlp(ctx, 0, LENGTH_SCALE)
    Xs, Ts, Gs = [], [], []
    for sd in seeds:
        sc = scenes.tiny_scene(sd)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.seeded(ctx, scene, sd, per_pair, order_lo, order_hi)
        out = fpt.solve(ctx, scene, batch)
        X, G = net.features(scene, batch, with_gram=True)
        keep = (out["status"] & fpt.ST_SOLVED) > 0
        T = torch.zeros((batch.n_paths, 4, 2), dtype=torch.float32, device=X.device)
        m = min(4, batch.n_max)
        T[:, :m] = out["T"][:, :m]
        Xs.append(X[keep])
        Ts.append(T[keep].reshape(-1, 8))
        Gs.append(G[keep])
    return torch.cat(Xs).contiguous(), torch.cat(Ts).contiguous(), torch.cat(Gs).contiguous()


def train(ctx, X, T, G, epochs=3, batch=8192, lr=1e-3, lr_decay=0.5, seed=0, log=None):
    """Adam on shuffled mini-batches (fpt_mlp_train: the schedule runs in the library); returns the network
    and the per-epoch mean batch loss."""
    net = fpt.Mlp(ctx, seed, LENGTH_SCALE)
    history = net.train(X, T, G, epochs, batch=batch, lr=lr, lr_decay=lr_decay, seed=seed)
    if log:
        for ep, v in enumerate(history):
            log(f"epoch {ep}: loss {v:.5f}")
    return net, history


def evaluate(ctx, net, seeds=EVAL_SEEDS, per_pair=1_000_000, order_lo=1, order_hi=4, max_iters=32, repeats=3):
    """Plain vs learned start on unseen scenes: iterations, solved paths, device time (solve + backward)."""
    import torch

    net.attach()
    res = {}
    for mode in (0, 1):
        p = fpt.default_params(init_mode=mode, max_iters=max_iters)
        tot_ms = 0.0
        solved = paths = iters = 0
        rho_max = 0.0
        for sd in seeds:
            sc = scenes.tiny_scene(sd)
            scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
            batch = fpt.Batch.seeded(ctx, scene, sd + 7, per_pair, order_lo, order_hi)
            out = fpt.alloc_outputs(ctx, batch, with_X=False)
            m = fpt.ST_VALID | fpt.ST_SOLVED
            fpt.solve(ctx, scene, batch, p, out)  # buckets the batch, warms up
            ctx.sync()
            stream = torch.cuda.current_stream()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(repeats):
                fpt.solve_grad(ctx, scene, batch, p, dL_status_mask=m, out=out)
            b.record(stream)
            torch.cuda.synchronize()
            tot_ms += a.elapsed_time(b) / repeats
            st = out["status"]
            s = (st & fpt.ST_SOLVED) > 0
            solved += int(s.sum())
            paths += batch.n_paths
            run = (st & (fpt.ST_REPEAT | fpt.ST_INVALID_INPUT)) == 0
            iters += int(out["iters"][run].to(torch.int64).sum())
            if bool(s.any()):
                rho_max = max(rho_max, float(out["rho"][s].max()))
        res["learned" if mode else "plain"] = {
            "solves_per_s": solved / (tot_ms / 1e3), "solved": solved, "paths": paths,
            "mean_bfgs_iters": iters / max(1, paths), "ms_solve_backward": tot_ms, "max_rho_solved_m": rho_max}
    return res


def run(ctx, per_pair_train=200_000, per_pair_eval=1_000_000, epochs=3, log=None):
    t0 = time.perf_counter()
    X, T, G = make_dataset(ctx, per_pair=per_pair_train)
    t1 = time.perf_counter()
    net, hist = train(ctx, X, T, G, epochs=epochs, log=log)
    t2 = time.perf_counter()
    ev = evaluate(ctx, net, per_pair=per_pair_eval)
    ev["train_samples"] = int(X.shape[0])
    ev["train_loss_per_epoch"] = hist
    ev["data_s"], ev["train_s"] = t1 - t0, t2 - t1
    return net, ev
