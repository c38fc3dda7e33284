"""Pins for the oracle's line MLP (CPU): gradient against central
differences of the loss, GELU against its closed forms, Adam against a
hand-computed first step, and the feature / scatter maps against
direct per-line loops."""
import math

import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from oracle import mlp as M
from oracle.mesh import line_nodes
from oracle.rules import Rules


def test_gelu_closed_forms():
    x = np.linspace(-6, 6, 101)
    assert np.allclose(M.gelu(x), 0.5 * x * (1 + np.tanh(math.sqrt(2 / math.pi) * (x + 0.044715 * x ** 3))))
    assert abs(M.gelu(np.array([0.0]))[0]) == 0.0
    assert np.allclose(M.gelu(np.array([20.0])), 20.0) and abs(M.gelu(np.array([-20.0]))[0]) < 1e-12
    h = 1e-6
    assert np.allclose(M.gelu_prime(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h), atol=1e-8)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    n_in, n_out, hid = 7, 3, 6
    theta = M.init_params(n_in, n_out, seed=1, hidden=hid) + 0.1 * rng.standard_normal(M.n_params(n_in, n_out, hid))
    X = rng.standard_normal((9, n_in))
    T = rng.standard_normal((9, n_out))
    _, g = M.loss_and_grad(theta, X, T, hidden=hid)
    fd = np.zeros_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = 1e-6
        fd[k] = (M.loss_and_grad(theta + e, X, T, hid)[0] - M.loss_and_grad(theta - e, X, T, hid)[0]) / 2e-6
    assert np.abs(g - fd).max() < 1e-8 * max(1.0, np.abs(fd).max())


def test_adam_first_step():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    th, m, v = M.adam_update(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # with bias correction the first step moves each weight by lr * sign(g)
    assert np.allclose(th, theta - 0.01 * np.sign(g) * (np.abs(g) / (np.abs(g) + 1e-8)))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_n_params_of_the_configured_network():
    # 69 -> 128 -> 128 -> 128 -> 20
    assert M.n_params(69, 20) == 69 * 128 + 128 + 2 * (128 * 128 + 128) + 128 * 20 + 20 == 44564


def test_features_targets_and_scatter_follow_the_lines():
    m = I.tgv_mesh(2, 3)
    D, p = 3, 3
    rng = np.random.default_rng(4)
    U = [rng.standard_normal((8, 5, 64)) for _ in range(4)]
    F = M.line_state_features(U[2], U[1], U[0], D, p)
    nl = 16
    for e in (0, 5):
        for l in (0, 7, 15):
            ln = line_nodes(D, p, 0, l)
            row = F[e * nl + l]
            for t, a in enumerate(ln):
                assert np.allclose(row[t * 5:(t + 1) * 5], U[2][e, :, a])
                assert np.allclose(row[20 + t * 5:20 + (t + 1) * 5], U[2][e, :, a] - U[1][e, :, a])
                assert np.allclose(row[40 + t * 5:40 + (t + 1) * 5], U[1][e, :, a] - U[0][e, :, a])
    Tg = M.line_targets(U[3], U[2], U[1], D, p)
    back = M.scatter_correction(Tg, U[2], U[1], D, p)
    assert np.allclose(back, U[3])
    G = M.line_metric_features(m, Rules(p, m["s"]))
    assert G.shape == (8 * 16, 9)
    # near-identity map: G / h close to the identity
    assert np.allclose(G.reshape(-1, 3, 3).mean(axis=0), np.eye(3), atol=0.1)
