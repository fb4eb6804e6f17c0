"""Pins of the warm-start network's CPU reference (oracle/mlp_oracle.py).

The gradient is checked against central finite differences (which never use
the backward formulas), a one-layer network against its closed form, and
Adam against values worked by hand.  Planted mistakes must be caught.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _fd_grad(params, widths, X, T, w, h=1e-6):
    g = np.zeros_like(params)
    for i in range(params.size):
        e = np.zeros_like(params)
        e[i] = h
        lp, _ = M.loss_and_grad(params + e, widths, X, T, w)
        lm, _ = M.loss_and_grad(params - e, widths, X, T, w)
        g[i] = (lp - lm) / (2 * h)
    return g


@pytest.mark.parametrize("widths", [[3, 4], [3, 5, 2], [4, 6, 5, 3]])
def test_gradient_matches_central_differences(widths):
    rng = np.random.default_rng(len(widths))
    p = rng.standard_normal(M.param_count(widths)) * 0.7
    X = rng.standard_normal((5, widths[0]))
    T = rng.standard_normal((5, widths[-1]))
    w = rng.uniform(0.5, 2.0, widths[-1])
    _, g = M.loss_and_grad(p, widths, X, T, w)
    assert np.allclose(g, _fd_grad(p, widths, X, T, w), rtol=1e-6, atol=1e-7)


def test_one_layer_is_least_squares():
    # a single linear layer: loss = ||X W + b - T||^2 / B, gradient 2/B [X 1]'(XW + b - T)
    rng = np.random.default_rng(1)
    X, T = rng.standard_normal((7, 3)), rng.standard_normal((7, 2))
    p = rng.standard_normal(M.param_count([3, 2]))
    W, b = p[:6].reshape(3, 2), p[6:]
    R = X @ W + b - T
    loss, g = M.loss_and_grad(p, [3, 2], X, T)
    assert loss == pytest.approx(np.sum(R * R) / 7, rel=1e-14)
    assert np.allclose(g[:6].reshape(3, 2), 2 / 7 * X.T @ R, rtol=1e-13)
    assert np.allclose(g[6:], 2 / 7 * R.sum(axis=0), rtol=1e-13)
    # at the least-squares solution the gradient vanishes
    Xa = np.hstack([X, np.ones((7, 1))])
    sol = np.linalg.lstsq(Xa, T, rcond=None)[0]
    p_star = np.concatenate([sol[:3].ravel(), sol[3]])
    assert np.allclose(M.loss_and_grad(p_star, [3, 2], X, T)[1], 0.0, atol=1e-12)


def test_relu_blocks_the_gradient_of_inactive_units():
    # hidden unit 0 always negative: its incoming weights get no gradient
    widths = [2, 2, 1]
    p = np.zeros(M.param_count(widths))
    W1 = np.array([[-1.0, 1.0], [-1.0, 1.0]])
    p[:4] = W1.ravel()
    p[4:6] = [-0.5, 0.1]
    p[6:8] = [3.0, 2.0]
    X = np.abs(np.random.default_rng(2).standard_normal((4, 2)))
    _, g = M.loss_and_grad(p, widths, X, np.ones((4, 1)))
    assert g[0] == 0.0 and g[2] == 0.0 and g[4] == 0.0 and g[6] == 0.0
    assert g[1] != 0.0 and g[5] != 0.0


def test_adam_first_steps_by_hand():
    opt = M.Adam(2, lr=0.1)
    p = np.array([1.0, -2.0])
    g = np.array([0.5, -4.0])
    p1 = opt.step(p, g)
    # step 1: m_hat = g, v_hat = g^2 -> p - lr * sign(g) (up to eps)
    assert np.allclose(p1, p - 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-15)
    g2 = np.array([1.0, 0.0])
    p2 = opt.step(p1, g2)
    m = 0.9 * 0.1 * g + 0.1 * g2
    v = 0.999 * 0.001 * g * g + 0.001 * g2 * g2
    mh, vh = m / (1 - 0.9 ** 2), v / (1 - 0.999 ** 2)
    assert np.allclose(p2, p1 - 0.1 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-14)


def test_training_reduces_the_loss_of_a_planted_map():
    rng = np.random.default_rng(3)
    widths = [4, 16, 3]
    X = rng.standard_normal((64, 4))
    T = np.maximum(X @ rng.standard_normal((4, 3)), 0) + 0.1
    p = M.he_init(widths, 0)
    opt = M.Adam(p.size, lr=1e-2)
    l0, _ = M.loss_and_grad(p, widths, X, T)
    for _ in range(300):
        _, g = M.loss_and_grad(p, widths, X, T)
        p = opt.step(p, g)
    l1, _ = M.loss_and_grad(p, widths, X, T)
    assert l1 < 0.05 * l0


def test_planted_backward_mistakes_are_caught(monkeypatch):
    widths = [3, 5, 2]
    rng = np.random.default_rng(4)
    p = rng.standard_normal(M.param_count(widths))
    X, T = rng.standard_normal((6, 3)), rng.standard_normal((6, 2))
    fd = _fd_grad(p, widths, X, T, None)
    real_forward = M.forward

    def no_mask(params, widths_, X_):  # a "ReLU" whose mask is dropped in backward
        out, zs, acts = real_forward(params, widths_, X_)
        return out, [np.abs(z) + 1.0 for z in zs], acts

    monkeypatch.setattr(M, "forward", no_mask)
    _, g = M.loss_and_grad(p, widths, X, T)
    assert not np.allclose(g, fd, rtol=1e-4, atol=1e-6)
