"""CPU FP64 reference of the warm-start network (test infrastructure only).

Only tests/ and bench.py's CPU legs import this module; the product path
never does.  The network is the one the learned warm start uses: a
multilayer perceptron with ReLU after every layer but the last,

    a_0 = input,   z_l = a_{l-1} W_l + b_l,   a_l = relu(z_l) (l < L),  out = z_L,

W_l of shape (width_{l-1}, width_l) and rows as samples, trained on the
weighted squared error

    loss = (1/B) sum_r sum_j w_j (out_rj - target_rj)^2

with the Adam update (Kingma and Ba, 2015: moments with beta1, beta2, bias
correction, step lr * m_hat / (sqrt(v_hat) + eps)).  Parameters are packed in
layer order, each layer as W (row-major) then b.

The gradient here is the chain rule written out layer by layer; the pins in
tests/test_mlp_oracle_pins.py check it against central finite differences,
which do not use it.
"""
from __future__ import annotations

import numpy as np


def param_count(widths) -> int:
    return int(sum(widths[i] * widths[i + 1] + widths[i + 1] for i in range(len(widths) - 1)))


def unpack(params: np.ndarray, widths):
    """[(W_1, b_1), ..., (W_L, b_L)] views into the packed vector."""
    out, o = [], 0
    for i in range(len(widths) - 1):
        a, b = widths[i], widths[i + 1]
        W = params[o:o + a * b].reshape(a, b)
        o += a * b
        bias = params[o:o + b]
        o += b
        out.append((W, bias))
    return out


def forward(params: np.ndarray, widths, X: np.ndarray):
    """Returns (output, [z_1..z_L], [a_0..a_{L-1}])."""
    layers = unpack(np.asarray(params, np.float64), widths)
    a = np.asarray(X, np.float64)
    zs, acts = [], [a]
    for i, (W, b) in enumerate(layers):
        z = a @ W + b
        zs.append(z)
        if i < len(layers) - 1:
            a = np.maximum(z, 0.0)
            acts.append(a)
    return zs[-1], zs, acts


def loss_and_grad(params: np.ndarray, widths, X: np.ndarray, T: np.ndarray, w=None):
    """Weighted squared error (see module docstring) and its gradient."""
    out, zs, acts = forward(params, widths, X)
    B = X.shape[0]
    wv = np.ones(out.shape[1]) if w is None else np.asarray(w, np.float64)
    diff = out - np.asarray(T, np.float64)
    loss = float(np.sum(wv * diff * diff) / B)
    g = (2.0 / B) * wv * diff          # d loss / d out
    grads = []
    L = len(zs)
    for i in range(L - 1, -1, -1):
        a_prev = acts[i]
        gW = a_prev.T @ g
        gb = g.sum(axis=0)
        grads.append((gW, gb))
        if i > 0:
            W, _ = unpack(np.asarray(params, np.float64), widths)[i]
            g = (g @ W.T) * (zs[i - 1] > 0.0)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


class Adam:
    """Adam (Kingma and Ba, 2015) on a packed parameter vector."""

    def __init__(self, n: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, params: np.ndarray, grad: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        m_hat = self.m / (1.0 - self.b1 ** self.t)
        v_hat = self.v / (1.0 - self.b2 ** self.t)
        return params - self.lr * m_hat / (np.sqrt(v_hat) + self.eps)


def he_init(widths, seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, packed."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(widths) - 1):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / widths[i]), widths[i] * widths[i + 1]))
        parts.append(np.zeros(widths[i + 1]))
    return np.concatenate(parts)
