"""Host-side checks of the seeded generators (no GPU, no solver arithmetic)."""
import numpy as np

from paper_2405_16160_b300 import workloads as W


def test_portfolio_instance_shape_and_strict_feasibility():
    for i in range(5):
        p = W.portfolio(0, i)
        s = p.meta["sectors"]
        assert 20 <= p.n <= 400 and p.k == max(p.n // 10, 1) and 5 <= s <= 20
        assert p.m == 1 + p.n + s and p.m_eq == 1
        inst = p.to_instance()
        A = inst.scipy_A()
        x = np.full(p.n, 1.0 / p.n)
        r = A @ x - p.b
        assert abs(r[0]) < 1e-12                   # budget row, equality
        assert np.all(r[1:1 + p.n] < 0)            # long-only, strictly
        nonempty = np.asarray(abs(A[1 + p.n:]).sum(axis=1)).ravel() > 0
        assert np.all(r[1 + p.n:][nonempty] < 0)  # sector caps, strictly


def test_portfolio_substreams_do_not_depend_on_the_batch():
    a = W.portfolio_batch(2, count=6)
    b = W.portfolio_batch(2, count=3)
    for p, q in zip(a[:3], b):
        assert p.n == q.n and np.array_equal(p.F, q.F) and np.array_equal(p.c, q.c)


def test_low_rank_q_is_written_out_exactly():
    p = W.portfolio(1, 0, 20, 30)
    Q = p.to_instance().scipy_Q().toarray()
    assert np.allclose(Q, p.F @ p.F.T + np.diag(p.qd), rtol=0, atol=1e-15)
    assert np.allclose(Q, Q.T) and np.linalg.eigvalsh(Q).min() > 0


def test_portfolio_family_perturbs_a_shared_base():
    fam = W.portfolio_family(0, seeds=[1, 2])
    f, g = fam
    assert (f.n, f.m, f.k) == (2000, 2031, 50)
    assert np.array_equal(f.qd, g.qd) and np.array_equal(f.A_col, g.A_col)
    d = f.F - g.F  # two independent perturbations of std 0.1/sqrt(k)
    assert abs(d.std() - np.sqrt(2) * 0.1 / np.sqrt(50)) < 0.002


def test_portfolio_bounds_form_drops_only_the_long_only_rows():
    for i in range(3):
        p, q = W.portfolio(0, i), W.portfolio(0, i, bounds=True)
        s = p.meta["sectors"]
        assert q.m == 1 + s and q.m_eq == 1 and np.array_equal(p.F, q.F)
        assert np.array_equal(p.c, q.c) and np.array_equal(p.qd, q.qd)
        Ap = p.to_instance().scipy_A().toarray()
        Aq = q.to_instance().scipy_A().toarray()
        keep = np.r_[0, np.arange(1 + p.n, p.m)]
        assert np.array_equal(Ap[keep], Aq) and np.array_equal(p.b[keep], q.b)
        assert np.array_equal(Ap[1:1 + p.n], -np.eye(p.n)) and np.all(p.b[1:1 + p.n] == 0)
        assert np.all(q.lo == 0) and np.all(np.isinf(q.hi))
        inst = q.to_instance()
        assert inst.lo is q.lo and inst.hi is q.hi
    assert p.lo is None and p.to_instance().lo is None


def test_portfolio_family_bounds_form_shares_its_draws():
    fam = W.portfolio_family(0, seeds=[3], n=200, k=10, sectors=8)
    fb = W.portfolio_family(0, seeds=[3], n=200, k=10, sectors=8, bounds=True)
    p, q = fam[0], fb[0]
    assert np.array_equal(p.F, q.F) and np.array_equal(p.c, q.c)
    assert (p.m, q.m) == (1 + 200 + 8, 1 + 8) and q.m_eq == 1
    assert np.all(q.lo == 0) and np.all(np.isinf(q.hi))


def test_cli_parses_its_options():
    import pytest
    from paper_2405_16160_b300 import solve as S
    with pytest.raises(SystemExit) as e:
        S.main(["--help"])
    assert e.value.code == 0
    with pytest.raises(SystemExit):
        S.main(["--workload", "no_such_workload"])


def test_warm_start_network_has_its_own_initializer():
    # the learned warm start's starting weights come from the package, not
    # from the CPU checker: He-normal (std sqrt(2 / fan_in)) weights and zero
    # biases, packed per layer as W then b, float32, and fit() defaults to it
    import inspect

    from paper_2405_16160_b300 import warmstart as WS

    widths = [300, 200, 50]
    p = WS.he_normal_params(widths, 3)
    assert p.dtype == np.float32
    assert p.size == sum(a * b + b for a, b in zip(widths[:-1], widths[1:]))
    o = 0
    for a, b in zip(widths[:-1], widths[1:]):
        W_, bias = p[o:o + a * b], p[o + a * b:o + a * b + b]
        o += a * b + b
        assert np.all(bias == 0)
        assert abs(W_.std() / np.sqrt(2.0 / a) - 1.0) < 0.05
        assert abs(W_.mean()) < 5 * np.sqrt(2.0 / a) / np.sqrt(a * b)
    assert np.array_equal(p, WS.he_normal_params(widths, 3))
    assert not np.array_equal(p, WS.he_normal_params(widths, 4))
    assert inspect.signature(WS.WarmStartModel.fit).parameters["init"].default is WS.he_normal_params


def test_split_prediction_is_the_per_instance_projection():
    """The batch's packed warm start from the network's outputs: row i of
    the outputs gives x_i = max(p[:n] / n, 0) and y_i = p[n:] * Y_SCALE with
    the inequality rows (after the first m_eq) projected onto y >= 0,
    instance after instance."""
    from paper_2405_16160_b300 import warmstart as WS
    rng = np.random.default_rng(4)
    count, n, m, m_eq = 6, 9, 5, 2
    pred = rng.normal(size=(count, n + m)).astype(np.float32)
    x0, y0 = WS.split_prediction(pred, n, m_eq)
    assert x0.shape == (count * n,) and y0.shape == (count * m,)
    for i in range(count):
        p = pred[i].astype(np.float64)
        xi = np.array([max(v / n, 0.0) for v in p[:n]])
        yi = np.array([v * WS.Y_SCALE if r < m_eq else max(v * WS.Y_SCALE, 0.0)
                       for r, v in enumerate(p[n:])])
        assert np.array_equal(x0[i * n:(i + 1) * n], xi)
        assert np.array_equal(y0[i * m:(i + 1) * m], yi)
