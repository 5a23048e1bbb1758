"""Pins of the FP64 reference MLP: gradients against central finite
differences, the GELU derivative against differences of GELU, and one Adam
step against its closed form."""
import math

import numpy as np

import synth
from oracle.mlp import OracleMLP, gelu, gelu_grad


def _net(sizes=(5, 7, 6, 3), seed=11):
    W, b = [], []
    for l in range(len(sizes) - 1):
        W.append(synth.uniform_matrix(seed + l, sizes[l + 1], sizes[l], -0.6, 0.6))
        b.append(synth.uniform(seed + 50 + l, sizes[l + 1]) - 0.5)
    return OracleMLP(sizes, np.full(sizes[0], 1.0), np.full(sizes[0], 5.0),
                     np.linspace(0.9, 1.1, sizes[-1]), np.full(sizes[-1], 3.0), (W, b))


def test_gelu_closed_form_and_derivative():
    z = np.linspace(-6, 6, 241)
    assert abs(gelu(np.array(0.0))) == 0.0
    assert abs(gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15     # 1 * Phi(1)
    assert np.all(np.abs(gelu(z) - np.maximum(z, 0)) < 1e-6 + 0.2 * np.exp(-z * z / 8))
    h = 1e-6
    assert np.allclose(gelu_grad(z), (gelu(z + h) - gelu(z - h)) / (2 * h), atol=1e-8)


def test_gradients_match_finite_differences():
    net = _net()
    x = synth.uniform_matrix(21, 9, 5, 0.8, 1.2)
    y = synth.uniform_matrix(22, 9, 3, 0.9, 1.1)
    loss, gW, gb = net.loss_and_grads(x, y)
    h = 1e-6
    for l in range(3):
        for (i, j) in [(0, 0), (1, 2), (net.W[l].shape[0] - 1, net.W[l].shape[1] - 1)]:
            orig = net.W[l][i, j]
            net.W[l][i, j] = orig + h
            lp = net.loss_and_grads(x, y)[0]
            net.W[l][i, j] = orig - h
            lm = net.loss_and_grads(x, y)[0]
            net.W[l][i, j] = orig
            assert abs((lp - lm) / (2 * h) - gW[l][i, j]) < 1e-7 * max(1.0, abs(gW[l][i, j]))
        k = net.b[l].shape[0] - 1
        orig = net.b[l][k]
        net.b[l][k] = orig + h
        lp = net.loss_and_grads(x, y)[0]
        net.b[l][k] = orig - h
        lm = net.loss_and_grads(x, y)[0]
        net.b[l][k] = orig
        assert abs((lp - lm) / (2 * h) - gb[l][k]) < 1e-7 * max(1.0, abs(gb[l][k]))


def test_adam_first_step_closed_form():
    """After one step from zero moments, m_hat = g and v_hat = g^2, so each
    parameter moves by -lr * g / (|g| + eps)."""
    net = _net()
    x = synth.uniform_matrix(23, 4, 5, 0.8, 1.2)
    y = synth.uniform_matrix(24, 4, 3, 0.9, 1.1)
    W0 = [w.copy() for w in net.W]
    _, gW, gb = net.loss_and_grads(x, y)
    net.adam_step(gW, gb, lr=1e-3)
    for l in range(3):
        assert np.allclose(net.W[l] - W0[l], -1e-3 * gW[l] / (np.abs(gW[l]) + 1e-8), rtol=1e-12, atol=1e-18)


def test_prediction_undoes_output_normalization():
    net = _net()
    x = synth.uniform_matrix(25, 3, 5, 0.8, 1.2)
    t = net.forward(x)
    assert np.allclose(net.predict(x), t / 3.0 + np.linspace(0.9, 1.1, 3))
