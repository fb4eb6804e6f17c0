"""The learned warm start: a network that maps a portfolio instance's
parameters to a starting point for the batched solver.

``WarmStartMLP`` is the binding of qp_mlp_* (the network's forward and
backward passes and the Adam update run in libpdhcg.so's kernels).  The
functions below only move data: they assemble inputs and targets, call the
batched solver and the network, and split the outputs.

Input convention (part of the model): the instance's expected returns mu,
standardised with the family's law, (mu - 0.05) / 0.02.  Output convention:
(n x, y / Y_SCALE), so that the targets are of order one.  A prediction is
projected onto the sign constraints (x >= 0 for the long-only rows, y >= 0
on inequality rows) before it is used.  The model also carries the primal
weight to start from: the median of the final omega over its training
solves.  Cold-start PDHCG is the fallback: an instance the warm-started
solve leaves unsolved is solved again from zero.
"""
from __future__ import annotations

from ctypes import POINTER, byref, c_double, c_float, c_int32, c_void_p

import time

import numpy as np

from . import _lib as L
from .solver import QPBatch, QPOptions, QPSolver

Y_SCALE = 0.05


class WarmStartMLP:
    """The qp_mlp handle.  Tensors passed in are float32 CUDA tensors."""

    def __init__(self, widths, max_batch: int, torch_memory: bool = True):
        self.lib = L.load_library()
        self.widths = [int(w) for w in widths]
        self.max_batch = int(max_batch)
        self._keep = []
        ctx = QPSolver._torch_ctx(self) if torch_memory else None
        w = (c_int32 * len(self.widths))(*self.widths)
        h = c_void_p()
        L.check(self.lib.qp_mlp_create(byref(h), len(self.widths) - 1, w, self.max_batch,
                                       byref(ctx) if ctx is not None else None),
                "qp_mlp_create")
        self.h = h
        self._ctx = ctx

    @property
    def param_count(self) -> int:
        return int(self.lib.qp_mlp_param_count(self.h))

    def set_params(self, params: np.ndarray) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.param_count:
            raise ValueError(f"expected {self.param_count} parameters, got {p.size}")
        L.check(self.lib.qp_mlp_set_params(self.h, p.ctypes.data_as(POINTER(c_float))),
                "qp_mlp_set_params")

    def get_params(self) -> np.ndarray:
        p = np.empty(self.param_count, np.float32)
        L.check(self.lib.qp_mlp_get_params(self.h, p.ctypes.data_as(POINTER(c_float))),
                "qp_mlp_get_params")
        return p

    @staticmethod
    def _check(t, cols):
        import torch

        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.shape[-1] != cols:
            raise ValueError("expected a contiguous float32 CUDA tensor with "
                             f"{cols} columns")

    def forward(self, x):
        import torch

        self._check(x, self.widths[0])
        out = torch.empty((x.shape[0], self.widths[-1]), dtype=torch.float32, device=x.device)
        L.check(self.lib.qp_mlp_forward(self.h, int(x.shape[0]), c_void_p(x.data_ptr()),
                                        c_void_p(out.data_ptr())), "qp_mlp_forward")
        return out

    def loss_grad(self, x, target, w=None, want_grad: bool = False):
        import torch

        self._check(x, self.widths[0])
        self._check(target, self.widths[-1])
        g = (torch.empty(self.param_count, dtype=torch.float32, device=x.device)
             if want_grad else None)
        loss = c_double()
        L.check(self.lib.qp_mlp_loss_grad(
            self.h, int(x.shape[0]), c_void_p(x.data_ptr()), c_void_p(target.data_ptr()),
            c_void_p(w.data_ptr()) if w is not None else None,
            c_void_p(g.data_ptr()) if g is not None else None, byref(loss)), "qp_mlp_loss_grad")
        return loss.value, g

    def adam_step(self, lr: float) -> None:
        L.check(self.lib.qp_mlp_adam_step(self.h, c_float(lr)), "qp_mlp_adam_step")

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.qp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ pipeline
def features(insts) -> np.ndarray:
    """(count, n) float32 network inputs: standardised expected returns."""
    return np.stack([(-q.c - 0.05) / 0.02 for q in insts]).astype(np.float32)


def targets(xs, ys) -> np.ndarray:
    """(count, n + m) float32 network targets from solutions."""
    return np.stack([np.concatenate([x * x.size, y / Y_SCALE]) for x, y in zip(xs, ys)]
                    ).astype(np.float32)


def split_prediction(pred: np.ndarray, n: int, m_eq: int = 1):
    """Network outputs (one row per instance) -> the packed (x0, y0) of the
    batch in the solver's variables, instance after instance, projected onto
    x >= 0 and y >= 0 on the inequality rows (whole-array operations: a batch
    is thousands of instances)."""
    pred = np.asarray(pred, np.float64)
    x = np.maximum(pred[:, :n] / n, 0.0)
    y = pred[:, n:] * Y_SCALE
    y[:, m_eq:] = np.maximum(y[:, m_eq:], 0.0)
    return x.reshape(-1), y.reshape(-1)


def solve_family(insts, options: QPOptions | None = None, warm=None, phases=None, **overrides):
    """Solve instances with the batched solver (warm = (xs, ys) or None).
    Returns (results, xs, ys).  ``phases`` (a dict, optional) accumulates the
    wall seconds of create / set_warm_start and of results + solution, and
    the solve launch's device milliseconds."""
    t0 = time.perf_counter()
    with QPBatch(insts) as bt:
        o = options or QPOptions()
        for k, v in overrides.items():
            setattr(o, k, v)
        if warm is not None:
            bt.set_warm_start(*warm)
            o.warm_start = 1
        t1 = time.perf_counter()
        ms = bt.solve(o)
        t2 = time.perf_counter()
        res = bt.results()
        xs, ys = bt.solution()
        t3 = time.perf_counter()
    if phases is not None:
        for key, v in (("create_s", t1 - t0), ("solve_s", t2 - t1), ("solve_device_ms", ms),
                       ("fetch_s", t3 - t2)):
            phases[key] = phases.get(key, 0.0) + v
    return res, xs, ys


def solve_with_fallback(insts, warm, options: QPOptions | None = None, phases=None,
                        **overrides):
    """Warm-started batched solve; instances it leaves unsolved are solved
    again from the cold start.  Returns (results, xs, ys, n_fallback)."""
    res, xs, ys = solve_family(insts, options, warm=warm, phases=phases, **overrides)
    bad = [i for i, r in enumerate(res) if r["termination"] != L.TERM_SOLVED]
    if bad:
        res2, xs2, ys2 = solve_family([insts[i] for i in bad], options, phases=phases,
                                      **overrides)
        for j, i in enumerate(bad):
            res[i], xs[i], ys[i] = res2[j], xs2[j], ys2[j]
    return res, xs, ys, len(bad)


def train(net: WarmStartMLP, X: np.ndarray, T: np.ndarray, epochs: int, batch: int, lr: float,
          seed: int = 0, device: str = "cuda"):
    """Adam on the squared error over shuffled minibatches; returns the
    per-epoch mean loss.  The shuffling order comes from numpy's seeded
    generator."""
    import torch

    Xd = torch.as_tensor(X, device=device)
    Td = torch.as_tensor(T, device=device)
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        perm = torch.as_tensor(rng.permutation(X.shape[0]), device=device)
        tot, cnt = 0.0, 0
        for s in range(0, X.shape[0] - batch + 1, batch):
            idx = perm[s:s + batch]
            loss, _ = net.loss_grad(Xd[idx].contiguous(), Td[idx].contiguous())
            net.adam_step(lr)
            tot += loss
            cnt += 1
        hist.append(tot / max(cnt, 1))
    return hist


def predict(net: WarmStartMLP, X: np.ndarray, n: int, device: str = "cuda", m_eq: int = 1):
    """The packed (x0, y0) of split_prediction for the rows of X, formed on
    the device from the network's outputs (the same operations, in FP64) and
    copied to the host once."""
    import torch

    xs, ys = [], []
    for s in range(0, X.shape[0], net.max_batch):
        pred = net.forward(torch.as_tensor(X[s:s + net.max_batch], device=device)
                           .contiguous()).double()
        x = torch.clamp(pred[:, :n] / n, min=0.0)
        y = pred[:, n:] * Y_SCALE
        y[:, m_eq:] = torch.clamp(y[:, m_eq:], min=0.0)
        xs.append(x.reshape(-1))
        ys.append(y.reshape(-1))
    return torch.cat(xs).cpu().numpy(), torch.cat(ys).cpu().numpy()


def he_normal_params(widths, seed: int = 0) -> np.ndarray:
    """Starting parameters of the network, packed as qp_mlp expects (per layer
    W row-major, then b): weights drawn from N(0, 2 / fan_in) by a seeded
    PCG64 stream (He et al., 2015, for ReLU layers), biases zero; float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chunks = []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        w = rng.standard_normal(fan_in * fan_out) * np.sqrt(2.0 / fan_in)
        chunks += [w.astype(np.float32), np.zeros(fan_out, np.float32)]
    return np.concatenate(chunks)


class WarmStartModel:
    """A trained network plus the family's starting primal weight."""

    def __init__(self, net: WarmStartMLP, n: int, omega0: float):
        self.net, self.n, self.omega0 = net, n, float(omega0)

    @classmethod
    def fit(cls, insts, results, xs, ys, hidden=(512, 512), epochs: int = 100, batch: int = 128,
            lr: float = 1e-3, seed: int = 0, init=he_normal_params):
        """Train on solved instances; ``init(widths, seed)`` gives the packed
        starting parameters (default: he_normal_params)."""
        X, T = features(insts), targets(xs, ys)
        widths = [X.shape[1], *hidden, T.shape[1]]
        net = WarmStartMLP(widths, max_batch=max(batch, 256))
        net.set_params(np.asarray(init(widths, seed), dtype=np.float32))
        hist = train(net, X, T, epochs=epochs, batch=batch, lr=lr, seed=seed)
        omega0 = float(np.median([r["omega"] for r in results]))
        model = cls(net, X.shape[1], omega0)
        model.history = hist
        return model

    def propose(self, insts):
        """The packed (x0, y0) for the instances (QPBatch.set_warm_start)."""
        return predict(self.net, features(insts), self.n)

    def solve(self, insts, options: QPOptions | None = None, phases=None, **overrides):
        """Warm-started batched solve with the cold-start fallback."""
        t0 = time.perf_counter()
        warm = self.propose(insts)
        if phases is not None:
            phases["propose_s"] = phases.get("propose_s", 0.0) + time.perf_counter() - t0
        return solve_with_fallback(insts, warm, options, phases=phases, omega0=self.omega0,
                                   **overrides)
