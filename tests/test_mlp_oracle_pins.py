"""Pins of the FP64 warm-start network reference (CPU only)."""

import numpy as np
import pytest

from oracle import mlp_oracle as mo
from paper_2510_16172_gb300 import scenes


def small_params(seed=0):
    rng = np.random.default_rng(seed)
    P = {}
    for name, shape in mo.SIZES:
        fan_in = shape[1] if len(shape) == 2 else 1
        P[name] = rng.uniform(-1, 1, shape) / np.sqrt(fan_in) if len(shape) == 2 else 0.1 * rng.standard_normal(shape)
    P["W4"][8:] = 0.0
    P["b4"][8:] = 0.0
    return mo.pack(P)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([np.random.default_rng(1).standard_normal(10000) * 10.0 ** np.arange(-3, 3).repeat(1667)[:10000],
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mo.bf16(x), ref)


def test_gelu_matches_torch_and_its_derivative_fd():
    torch = pytest.importorskip("torch")
    z = np.linspace(-6, 6, 241)
    ref = torch.nn.functional.gelu(torch.tensor(z, dtype=torch.float64), approximate="tanh").numpy()
    np.testing.assert_allclose(mo.gelu(z), ref, atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(mo.gelu_grad(z), (mo.gelu(z + h) - mo.gelu(z - h)) / (2 * h), atol=1e-8)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = small_params(3)
    B = 12
    X = rng.standard_normal((B, 64)) * 0.5
    for s in range(4):  # slot activity flags
        X[:, 6 + 11 * s] = (rng.uniform(size=B) < 0.7).astype(float)
    T = rng.standard_normal((B, 8))
    a = rng.standard_normal((B, 4, 2, 3)) * (rng.uniform(size=(B, 4, 1, 1)) < 0.7)
    G = np.stack([np.sum(a[:, :, 0] * a[:, :, 0], -1), np.sum(a[:, :, 0] * a[:, :, 1], -1),
                  np.sum(a[:, :, 1] * a[:, :, 1], -1)], axis=2)
    loss, g = mo.loss_grad(params, X, T, G, round_bf16=False)
    h = 1e-6
    idx = rng.choice(mo.N_PARAMS, 60, replace=False)
    for k in idx:
        p1, p2 = params.copy(), params.copy()
        p1[k] += h
        p2[k] -= h
        fd = (mo.loss_grad(p1, X, T, G, False)[0] - mo.loss_grad(p2, X, T, G, False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_loss_definition_on_a_hand_example():
    """One quad slot with a1 = (2,0,0)/S, a2 = (0,3,0)/S: world error (2 dy0, 3 dy1, 0)."""
    G = np.zeros((1, 4, 3))
    G[0, 0] = [4.0, 0.0, 9.0]
    Y = np.zeros((1, 16))
    Y[0, 0], Y[0, 1] = 0.5, 0.25
    T = np.zeros((1, 8))
    loss, dY = mo.loss_and_dY(G, Y, T)
    assert loss == pytest.approx(1.0 + 0.5625)
    assert dY[0, 0] == pytest.approx(2 * 2 * 1.0) and dY[0, 1] == pytest.approx(2 * 3 * 0.75)
    loss0, _ = mo.loss_and_dY(G, np.zeros((1, 16)), T)
    assert loss0 == 0.0


def test_features_of_a_hand_example():
    """Plane z = 0 spanned by (2,0,0), (0,4,0) from the origin; edge along z at (1,1); TX (0,0,10), RX (10,0,10)."""
    types = np.array([0, 1], np.uint8)
    verts = np.array([[[0, 0, 0], [2, 0, 0], [0, 4, 0]], [[1, 1, 1], [1, 1, 5], [0, 0, 0]]], float)
    sc = scenes.Scene(types, verts, np.array([[0.0, 0, 10]]), np.array([[10.0, 0, 10]]))
    F, G = mo.features(sc, np.array([[0, 1]]), np.array([2]), np.array([0]), np.array([0]), 10.0)
    o = np.array([5.0, 0, 10])
    np.testing.assert_allclose(F[0, 0:6], np.concatenate([([0, 0, 10] - o) / 10, ([10, 0, 10] - o) / 10]))
    # plane: projections (0,0,0) -> tau (0,0) and (10,0,0) -> tau (5,0); both 1 m (10 m / S) away
    np.testing.assert_allclose(F[0, 6:17], [1, 0, 0, 0, 5, 0, 1, 1, 0.2, 2.5, 0], atol=1e-12)
    # edge e0 = (1,1,1), a1 = (0,0,4): TX projects to z = 10 -> tau 9/4, RX too; distances sqrt(2)/10, sqrt(82)/10
    d_tx, d_rx = np.sqrt(2) / 10, np.sqrt(82) / 10
    np.testing.assert_allclose(F[0, 17:28], [1, 1, 2.25, 0, 2.25, 0, d_tx, d_rx, 0.4, 2.25, 0], atol=1e-12)
    assert np.all(F[0, 28:] == 0)
    np.testing.assert_allclose(G[0, 0], [0.04, 0.0, 0.16])
    np.testing.assert_allclose(G[0, 1], [0.16, 0.0, 0.0])
    assert np.all(G[0, 2:] == 0)
