"""Pins of the FP64 MLP oracle (forward, MSE gradient, Adam).

GELU against its erf definition evaluated independently (math.erf), its
derivative and the whole backpropagated gradient against central finite
differences, forward on a network whose weights vanish (closed form), and
Adam under a constant gradient, where every bias-corrected step has the
closed form p_t = p_0 - t lr g / (|g| + eps)."""

import math

import numpy as np
import pytest

import oracle as O


def test_gelu_matches_erf_definition_and_derivative():
    for z in (-4.0, -1.3, -0.2, 0.0, 0.5, 2.7):
        assert abs(O.gelu(z) - 0.5 * z * (1 + math.erf(z / math.sqrt(2)))) <= 1e-15 * max(1, abs(z))
        h = 1e-6
        fd = (O.gelu(z + h) - O.gelu(z - h)) / (2 * h)
        assert abs(O.gelu_grad(z) - fd) < 1e-8
    assert O.gelu(-40.0) == 0.0 or abs(O.gelu(-40.0)) < 1e-300
    assert abs(O.gelu(40.0) - 40.0) < 1e-12


@pytest.mark.parametrize("dims", [(3, 5, 4, 2), (30, 8, 8, 6), (2, 7, 1)])
def test_gradient_matches_central_finite_differences(dims):
    rng = np.random.default_rng(sum(dims))
    npar = O.mlp_param_count(dims)
    p = rng.normal(size=npar) * 0.5
    X = rng.normal(size=(7, dims[0]))
    T = rng.normal(size=(7, dims[-1]))
    loss, g = O.mlp_loss_grad(dims, p, X, T)
    Y = O.mlp_forward(dims, p, X)
    assert abs(loss - np.mean((Y - T) ** 2)) <= 1e-14 * loss
    idx = rng.choice(npar, size=min(npar, 60), replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp, _ = O.mlp_loss_grad(dims, pp, X, T)
        lm, _ = O.mlp_loss_grad(dims, pm, X, T)
        fd = (lp - lm) / (2 * h)
        assert abs(g[i] - fd) <= 1e-7 * max(1.0, abs(fd)), i


def test_forward_with_zero_weights_is_the_bias_chain():
    dims = (4, 3, 2)
    npar = O.mlp_param_count(dims)
    p = np.zeros(npar)
    b1 = np.array([0.3, -1.2, 2.0])
    W2 = np.array([[1.0, 2.0, -1.0], [0.5, 0.0, 3.0]])
    b2 = np.array([0.1, -0.2])
    o = 4 * 3
    p[o:o + 3] = b1
    p[o + 3:o + 3 + 6] = W2.ravel()
    p[o + 9:o + 11] = b2
    X = np.random.default_rng(0).normal(size=(5, 4))
    Y = O.mlp_forward(dims, p, X)
    g = np.array([0.5 * z * (1 + math.erf(z / math.sqrt(2))) for z in b1])
    assert np.allclose(Y, (W2 @ g + b2)[None, :].repeat(5, 0), rtol=0, atol=1e-15)


def test_adam_constant_gradient_closed_form():
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=9)
    g = rng.normal(size=9) * np.array([1e-3, 1, 10, 1e-6, 2, 3, 0.5, 1e2, 7])
    p, m, v = p0.copy(), np.zeros(9), np.zeros(9)
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        O.adam_step(p, g, m, v, t, lr=lr, eps=eps)
        exp = p0 - t * lr * g / (np.abs(g) + eps)
        assert np.allclose(p, exp, rtol=0, atol=1e-13)
