"""Ragged large batch: a 256-object city, 100,000,000 seeded sequences of order 1-5 (mixed
reflectors and edges), learned start, solve and implicit backward in one call.

Sampled paths are re-solved by the oracle (same tolerances as the other parity tests); the
gradients of the sum of valid solved lengths with respect to TX and RX are checked over all
paths against the envelope theorem (dL*/dTX = -u_0, dL*/dRX = u_n at a stationary path).
"""

import numpy as np
import pytest

import oracle
from paper_2510_16172_gb300 import fpt, scenes, warmstart

pytestmark = pytest.mark.gpu

PER_PAIR = 6_250_000  # x 16 RX = 100,000,000 paths


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    oracle.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


def test_city_100m_learned_start_solve_grad(ctx):
    import torch

    from test_gpu_parity import check_parity, oracle_solve

    # a network trained briefly on the solver's own tiny-scene solutions (its quality is not under test)
    X, T, G = warmstart.make_dataset(ctx, [21, 22], 20000)
    net = fpt.Mlp(ctx, 4, warmstart.LENGTH_SCALE)
    B = 4096
    n = X.shape[0] // B * B
    for step in range(100):
        k = (step * B) % n
        net.train_step(X[k:k + B], T[k:k + B], G[k:k + B], 1e-3, want_loss=False)
    net.attach()
    del X, T, G

    sc = scenes.city(0, n_rx=16)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    batch = fpt.Batch.seeded(ctx, scene, 5, PER_PAIR, 1, 5)
    assert batch.n_paths == 100_000_000
    mask = fpt.ST_VALID | fpt.ST_SOLVED
    out = fpt.alloc_outputs(ctx, batch, with_X=True)
    out, (g_tx, g_rx, g_v) = fpt.solve_grad(ctx, scene, batch, fpt.default_params(init_mode=1, max_iters=32),
                                            dL_status_mask=mask, out=out)
    ctx.sync()

    # sampled parity against the oracle
    rng = np.random.default_rng(11)
    gidx = np.sort(rng.choice(batch.n_paths, 3000, replace=False))
    gi = torch.as_tensor(gidx, device=out["T"].device)
    g = {k: v[gi].cpu().numpy() for k, v in out.items() if v is not None}
    ids, order, ti, ri = oracle.seeded_paths(sc, 5, PER_PAIR, 1, 5, gidx)
    ref = oracle_solve(sc, ids, order, ti, ri)
    check_parity(g, ref, min_solved_frac=0.99)

    # envelope theorem over every path: the gradient of sum(valid solved L) w.r.t. TX / RX
    st = out["status"]
    use = (st & mask) == mask
    assert int(use.sum()) > 0.01 * batch.n_paths  # random order-1..5 sequences: a few % valid and solved
    _, order_d, txi, rxi = fpt.enumerate(ctx, batch)
    dev = st.device
    tx = torch.as_tensor(sc.tx, device=dev)
    rx = torch.as_tensor(sc.rx, device=dev)
    e_tx = torch.zeros_like(tx)
    e_rx = torch.zeros_like(rx)
    step = 10_000_000
    for a in range(0, batch.n_paths, step):
        sl = slice(a, a + step)
        u = use[sl]
        Xs = out["X"][sl][u].double()
        o = order_d[sl][u].long()
        ti_s, ri_s = txi[sl][u].long(), rxi[sl][u].long()
        first = Xs[:, 0] - tx[ti_s]
        last = rx[ri_s] - Xs[torch.arange(Xs.shape[0], device=dev), o - 1]
        e_tx.index_add_(0, ti_s, -first / first.norm(dim=1, keepdim=True))
        e_rx.index_add_(0, ri_s, last / last.norm(dim=1, keepdim=True))
    assert torch.isfinite(g_v).all() and torch.isfinite(g_tx).all() and torch.isfinite(g_rx).all()
    scale = float(e_tx.abs().max())
    assert float((g_tx.double() - e_tx).abs().max()) <= 1e-4 * scale
    assert float((g_rx.double() - e_rx).abs().max()) <= 1e-4 * float(e_rx.abs().max())
