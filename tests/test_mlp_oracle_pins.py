"""Pins of the FP64 reference of the controller network (oracle/mlp_oracle.py)
to facts outside itself: textbook values of the normal CDF, the GELU
identities, central finite differences of the loss (independent of the
chain-rule code), the closed form of Adam's first step, and exact BF16 bit
patterns."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2609_19557_gb300 import mlp_data as D


def test_parameter_count_matches_layout():
    assert M.N_PARAMS == D.N_PARAMS == 5378


def test_gelu_textbook_values_and_identities():
    # GELU(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208 (normal tables)
    assert M.gelu(np.array(0.0)) == 0.0
    assert abs(M.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(M.gelu(np.array(2.0)) - 2 * 0.9772498680518208) < 1e-14
    z = np.linspace(-5, 5, 41)
    assert np.allclose(M.gelu(z) - M.gelu(-z), z, atol=1e-14)  # Phi(z) + Phi(-z) = 1
    assert abs(M.gelu_prime(np.array(0.0)) - 0.5) < 1e-15
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_prime(z), fd, rtol=1e-8, atol=1e-9)


def test_backward_matches_central_differences():
    theta = D.init_weights(3).astype(np.float64)
    theta[M.N_PARAMS - 2:] = [0.3, -0.2]  # nonzero output biases
    X = D.features(4, 5).astype(np.float64)
    T = np.random.default_rng(5).normal(size=(5, 2))
    w = np.array([1.0, 0.5, 2.0, 0.0, 1.5])
    Y, cache = M.forward(theta, X)
    _, dY = M.wmse(Y, T, w)
    g = M.backward(theta, cache, dY)
    rng = np.random.default_rng(6)
    idx = np.concatenate([rng.choice(M.N_PARAMS, 300, replace=False), np.arange(M.N_PARAMS - 2, M.N_PARAMS)])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss_of(tp, X, T, w) - M.loss_of(tm, X, T, w)) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, g[i], fd)


def test_wmse_gradient_and_value():
    Y = np.array([[1.0, 2.0], [0.0, -1.0]])
    T = np.array([[0.0, 2.0], [1.0, 1.0]])
    w = np.array([1.0, 3.0])
    L, dY = M.wmse(Y, T, w)
    assert abs(L - (1.0 * 1.0 + 3.0 * (1.0 + 4.0)) / 4.0) < 1e-15
    assert np.allclose(dY, 2 * w[:, None] * (Y - T) / 4.0)


def test_forward_special_cases():
    X = D.features(1, 7).astype(np.float64)
    p = {name: np.zeros(shp) for name, shp in M.SHAPES}
    p["b3"] = np.array([0.25, -4.0])
    Y, _ = M.forward(M.pack(p), X)
    assert np.array_equal(Y, np.tile(p["b3"], (7, 1)))  # no path from the inputs
    p["b2"] = np.linspace(-1, 1, 64)
    p["W3"] = np.ones((2, 64))
    Y, _ = M.forward(M.pack(p), X)
    assert np.allclose(Y, p["b3"] + M.gelu(p["b2"]).sum(), atol=1e-14)  # W2 = 0: constant hidden layer


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    t1, m, v = M.adam_step(th, g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    # bias-corrected m = g, v = g^2 at step 1: the step is lr * g / (|g| + eps)
    assert np.allclose(t1, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_bit_patterns():
    vals = np.array([1.0, -2.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, 0.0], dtype=np.float32)
    bits = D.bf16_bits(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1.0); 1 + 3*2^-8 ties up to 1 + 2^-6
    assert list(bits) == [0x3F80, 0xC000, 0x3F80, 0x3F82, 0x3F81, 0x0000]
    assert np.array_equal(D.bf16_values(bits), np.array([1, -2, 1, 1 + 2.0 ** -6, 1 + 2.0 ** -7, 0], np.float32))
