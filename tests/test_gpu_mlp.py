"""The warm-start network's kernels against the CPU FP64 reference
(oracle/mlp_oracle.py), and what the trained network gains.

FP32 kernels against FP64: forward and loss within 1e-5 relative, the
gradient within 1e-4 of its largest entry, Adam steps within 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as M
from oracle import pdhcg_oracle as O
from paper_2405_16160_b300 import _lib as L
from paper_2405_16160_b300 import warmstart as WS
from paper_2405_16160_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(widths, batch, seed):
    rng = np.random.default_rng(seed)
    p = M.he_init(widths, seed).astype(np.float32)
    X = rng.standard_normal((batch, widths[0])).astype(np.float32)
    T = rng.standard_normal((batch, widths[-1])).astype(np.float32)
    w = rng.uniform(0.5, 2.0, widths[-1]).astype(np.float32)
    return p, X, T, w


SHAPES = [([7, 33, 17, 5], 37), ([1, 1], 1), ([65, 64, 63], 129), ([2000, 128, 4031], 70)]


@pytest.mark.parametrize("widths,batch", SHAPES)
def test_forward_matches_oracle(widths, batch):
    p, X, _, _ = _case(widths, batch, 1)
    net = WS.WarmStartMLP(widths, max_batch=batch)
    net.set_params(p)
    got = net.forward(torch.as_tensor(X, device="cuda")).cpu().numpy()
    ref, _, _ = M.forward(p.astype(np.float64), widths, X.astype(np.float64))
    assert np.max(np.abs(got - ref)) <= 1e-5 * max(np.max(np.abs(ref)), 1.0)
    net.close()


@pytest.mark.parametrize("widths,batch", SHAPES)
def test_loss_and_gradient_match_oracle(widths, batch):
    p, X, T, w = _case(widths, batch, 2)
    net = WS.WarmStartMLP(widths, max_batch=batch)
    net.set_params(p)
    loss, g = net.loss_grad(torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda"),
                            torch.as_tensor(w, device="cuda"), want_grad=True)
    rl, rg = M.loss_and_grad(p.astype(np.float64), widths, X.astype(np.float64),
                             T.astype(np.float64), w.astype(np.float64))
    assert loss == pytest.approx(rl, rel=1e-5)
    g = g.cpu().numpy()
    assert np.max(np.abs(g - rg)) <= 1e-4 * np.max(np.abs(rg))
    net.close()


def test_adam_steps_match_oracle():
    widths, batch = [6, 20, 4], 16
    p, X, T, _ = _case(widths, batch, 3)
    net = WS.WarmStartMLP(widths, max_batch=batch)
    net.set_params(p)
    opt = M.Adam(p.size, lr=1e-2)
    q = p.astype(np.float64)
    Xd, Td = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    for _ in range(3):
        net.loss_grad(Xd, Td)
        net.adam_step(1e-2)
        _, g = M.loss_and_grad(q, widths, X.astype(np.float64), T.astype(np.float64))
        q = opt.step(q, g)
    assert np.max(np.abs(net.get_params() - q)) <= 1e-5 * max(np.max(np.abs(q)), 1.0)
    net.close()


def test_training_fits_a_planted_map():
    rng = np.random.default_rng(4)
    widths = [8, 64, 4]
    X = rng.standard_normal((512, 8)).astype(np.float32)
    T = np.maximum(X @ rng.standard_normal((8, 4)), 0).astype(np.float32)
    net = WS.WarmStartMLP(widths, max_batch=64)
    net.set_params(WS.he_normal_params(widths, 0))
    hist = WS.train(net, X, T, epochs=60, batch=64, lr=3e-3)
    assert hist[-1] < 0.05 * hist[0]
    net.close()


def test_learned_warm_start_cuts_iterations():
    # a small member of the parametric family: n = 200, k = 20, 10 sectors;
    # a start with relative error e saves about log(1/e) of the log(1/tol)
    # iterations of a linearly convergent method, so the gain is modest
    fam = W.portfolio_family(0, seeds=range(1, 1025 + 32), n=200, k=20, sectors=10)
    train_set, test_set = fam[:1024], fam[1024:]
    res, xs, ys = WS.solve_family(train_set, tol=1e-5, precision=L.PREC_MIXED)
    assert all(r["termination"] == L.TERM_SOLVED for r in res)
    model = WS.WarmStartModel.fit(train_set, res, xs, ys, hidden=(256, 256), epochs=40,
                                  batch=64)
    assert model.history[-1] < 0.5 * model.history[0]
    cold, _, _ = WS.solve_family(test_set, tol=1e-4, precision=L.PREC_MIXED)
    hot, xs_h, ys_h, n_fallback = model.solve(test_set, tol=1e-4, precision=L.PREC_MIXED)
    assert all(r["termination"] == L.TERM_SOLVED for r in hot) and n_fallback == 0
    for q, x, y in zip(test_set, xs_h, ys_h):  # the final KKT residual judges the result
        assert O.relkkt(O.problem_from_instance(q.to_instance()), x, y).relkkt <= 1e-4
    it_cold = np.mean([r["iterations"] for r in cold])
    it_hot = np.mean([r["iterations"] for r in hot])
    assert it_hot <= 0.95 * it_cold, (it_hot, it_cold)
    model.net.close()
