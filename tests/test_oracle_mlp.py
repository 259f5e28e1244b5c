"""Pins of the oracle's MLP (learned EOS guess): central finite differences of
the loss against the reverse-mode gradient, and the forward pass against a
numpy restatement built from matrix products."""
import numpy as np
import pytest


def init_params(seed):
    rng = np.random.default_rng(seed)
    H = 64
    parts = [rng.normal(0, 1 / np.sqrt(2), 2 * H), rng.normal(0, 0.1, H),
             rng.normal(0, 1 / np.sqrt(H), H * H), rng.normal(0, 0.1, H),
             rng.normal(0, 1 / np.sqrt(H), 2 * H), rng.normal(0, 0.1, 2)]
    return np.concatenate(parts)


def test_forward_matches_matrix_form(oracle):
    p = init_params(0)
    H = 64
    W1 = p[:128].reshape(H, 2); b1 = p[128:192]
    W2 = p[192:192 + 4096].reshape(H, H); b2 = p[4288:4352]
    W3 = p[4352:4480].reshape(2, H); b3 = p[4480:4482]
    x = np.random.default_rng(1).normal(size=(50, 2))
    silu = lambda a: a / (1 + np.exp(-a))
    y = silu(silu(x @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    assert np.allclose(oracle.mlp_forward(p, x), y, rtol=1e-13, atol=1e-13)


def test_gradient_central_differences(oracle):
    p = init_params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(16, 2))
    t = rng.normal(size=(16, 2))
    loss, g = oracle.mlp_loss_grad(p, x, t)
    idx = np.concatenate([np.arange(0, 4482, 37), [0, 127, 191, 4287, 4351, 4479, 4480, 4481]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, x, t)[0] - oracle.mlp_loss_grad(pm, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    y = oracle.mlp_forward(p, x)
    assert loss == pytest.approx(np.mean(np.sum((y - t) ** 2, axis=1)), rel=1e-14)
