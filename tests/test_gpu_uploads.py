"""Scene, endpoint and alphabet uploads are asynchronous on the context's stream.

The library builds its records on the host, keeps them until the scene (or batch) is
released and copies them on the context's stream, so a solve issued right after an upload
sees the new data, the caller may overwrite its host arrays as soon as the call returns, and
replacing a scene's endpoints gives the results of a scene built with the new ones.
"""

import numpy as np
import pytest

from paper_2510_16172_gb300 import fpt, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch

    from paper_2510_16172_gb300 import build

    build.build()
    assert torch.cuda.is_available()
    return fpt.Context(0)


def _solve(ctx, scene, lo=1, hi=3, alphabet=None):
    batch = fpt.Batch.exhaustive(ctx, scene, lo, hi, alphabet)
    out = fpt.solve(ctx, scene, batch)
    ctx.sync()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


def _same(a, b):
    for k in ("T", "X", "L", "status", "iters"):
        assert np.array_equal(a[k], b[k]), k


def test_host_arrays_may_change_after_the_upload(ctx):
    sc = scenes.tiny_scene(3, n_rx=2)
    ref = _solve(ctx, fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx))
    types, verts = sc.types.copy(), sc.verts.copy()
    tx, rx = sc.tx.copy(), sc.rx.copy()
    scene = fpt.Scene(ctx, types, verts, tx, rx)
    alphabet = np.arange(len(types), dtype=np.int32)
    batch = fpt.Batch.exhaustive(ctx, scene, 1, 3, alphabet)
    # overwrite every host input before anything is solved
    verts[:] = 0.0
    tx[:] = 1e3
    rx[:] = -1e3
    alphabet[:] = 0
    scene.verts[:] = 0.0
    out = fpt.solve(ctx, scene, batch)
    ctx.sync()
    _same({k: v.cpu().numpy() for k, v in out.items() if v is not None}, ref)


def test_replaced_endpoints_match_a_fresh_scene(ctx):
    sc = scenes.tiny_scene(4, n_rx=2)
    other = scenes.tiny_scene(5, n_rx=3)
    scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
    first = _solve(ctx, scene)
    scene.set_endpoints(other.tx, other.rx)  # the old device copies are freed, the new ones uploaded
    second = _solve(ctx, scene)
    _same(first, _solve(ctx, fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)))
    _same(second, _solve(ctx, fpt.Scene(ctx, sc.types, sc.verts, other.tx, other.rx)))
    assert second["L"].shape[0] == 3 * first["L"].shape[0] // 2


def test_back_to_back_scenes_without_synchronising(ctx):
    """Many scenes uploaded and solved in a row with no host synchronisation in between (the
    serving loop of the benchmark's end-to-end leg): every step gives its own scene's results."""
    import torch

    refs, outs, keep = [], [], []
    for seed in range(6):
        sc = scenes.tiny_scene(10 + seed, n_rx=2)
        refs.append(_solve(ctx, fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)))
    torch.cuda.synchronize()
    for seed in range(6):
        sc = scenes.tiny_scene(10 + seed, n_rx=2)
        scene = fpt.Scene(ctx, sc.types, sc.verts, sc.tx, sc.rx)
        batch = fpt.Batch.exhaustive(ctx, scene, 1, 3)
        outs.append(fpt.solve(ctx, scene, batch))
        keep.append((scene, batch))
    ctx.sync()
    for ref, out in zip(refs, outs):
        _same({k: v.cpu().numpy() for k, v in out.items() if v is not None}, ref)
