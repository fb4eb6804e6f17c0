"""Seeded synthetic QP instances shaped like the paper's workloads.

This module only draws random numbers and assembles CSR arrays.  It holds
none of the solver's arithmetic, so both the CUDA path and the CPU oracle can
be fed from it without sharing any of the method.

Problem form (paper Eq. (1)): min 1/2 x'Qx + c'x  s.t.  Ax <= b, Q PSD.
The first ``m_eq`` rows of A are equalities (the "Gx = q inside Ax <= b"
reading of the augmented-penalty paragraph of Section 4).

Instances
---------
``dense_small``  n=200, m=100 (the small latency-bound case):
    Q = D + M'M/50, D = diag U[0.1, 1], M 50x200 with Bernoulli(0.05) N(0,1)
    entries; A 100x200 with Bernoulli(0.05) N(0,1) entries; c ~ N(0,1);
    b = A x0 + s, x0 ~ N(0,1), s ~ U[0,1] (strictly feasible at x0).
``sparse_dd``  n=1e6, m=5e5 by default (the large sparse case):
    Q = diag(u) + S, u ~ U[0.5, 2]; S symmetric, every row draws 4 partners
    j != i uniformly with N(0, 0.1) values (std 0.1) and the pattern is
    mirrored (~8 off-diagonals per row); Q_ii = u_i + sum_j |S_ij| so Q is
    strictly diagonally dominant, hence positive definite.  A has exactly
    ``a_row_nnz`` (10) distinct uniform columns per row with N(0,1) values.
    c, b as above.  The same recipe at smaller n gives the parity cases.
``zipf_dd``  n=1e7, m=5e6 (the largest single QP):
    as ``sparse_dd`` with 2-3 partners per row (~5 nnz/row of Q) and A with
    8 distinct columns per row drawn from a Zipf(1.1) law over column ranks,
    mapped to columns by a seeded permutation.
``portfolio_batch``  4096 Markowitz-style QPs for the batched solver:
    instance i draws from the substream (seed, i): n ~ U{20..400}, k =
    floor(n/10) factors, F n x k with N(0, 1/k) entries (variance 1/k), Q =
    F F' + diag U[0.01, 0.1], c = -mu with mu ~ N(0.05, 0.02); A = the
    budget row 1'x = 1 (equality), long-only rows -x <= 0 and s ~ U{5..20}
    sector caps: every asset sits in one uniformly drawn sector j and
    sum_{i in S_j} x_i <= 1.5 |S_j| / n (so x = 1/n is strictly feasible).
``portfolio_family``  the parametric family of the learned warm start:
    n = 2000, k = 50, 30 sectors, budget and long-only rows (m = 2031); a
    base F0 and sector map from ``base_seed``, then per instance mu ~
    N(0.05, 0.02) and F = F0 + 0.1 * (1/sqrt(k)) * G with G ~ N(0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class QPInstance:
    """A QP in CSR form: min 1/2 x'Qx + c'x s.t. A x <= b (first m_eq rows =)."""

    n: int
    m: int
    m_eq: int
    Q_rowptr: np.ndarray  # int32 [n+1]
    Q_col: np.ndarray  # int32 [nnz_Q]
    Q_val: np.ndarray  # float64 [nnz_Q]
    A_rowptr: np.ndarray  # int32 [m+1]
    A_col: np.ndarray  # int32 [nnz_A]
    A_val: np.ndarray  # float64 [nnz_A]
    c: np.ndarray  # float64 [n]
    b: np.ndarray  # float64 [m]
    name: str = ""
    meta: dict = field(default_factory=dict)
    lo: np.ndarray | None = None  # variable bounds (+-inf where absent); None: none
    hi: np.ndarray | None = None

    @property
    def nnz_Q(self) -> int:
        return int(self.Q_rowptr[-1])

    @property
    def nnz_A(self) -> int:
        return int(self.A_rowptr[-1])

    def scipy_Q(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.Q_val, self.Q_col, self.Q_rowptr), shape=(self.n, self.n))

    def scipy_A(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.A_val, self.A_col, self.A_rowptr), shape=(self.m, self.n))


def _csr_arrays(M: sp.spmatrix):
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    return (M.indptr.astype(np.int32), M.indices.astype(np.int32),
            M.data.astype(np.float64))


def _bernoulli_normal(rng: np.random.Generator, rows: int, cols: int, density: float):
    mask = rng.random((rows, cols)) < density
    vals = rng.standard_normal((rows, cols))
    return np.where(mask, vals, 0.0)


def _feasible_rhs(rng, A: sp.csr_matrix, n: int, m_eq: int):
    x0 = rng.standard_normal(n)
    s = rng.random(A.shape[0])
    s[:m_eq] = 0.0  # equality rows hold exactly at x0
    return A @ x0 + s


def dense_small(seed: int = 0, n: int = 200, m: int = 100, k: int = 50,
                density: float = 0.05, m_eq: int = 0) -> QPInstance:
    """The n=200, m=100 instance (Q = D + M'M/50; A Bernoulli(0.05) N(0,1))."""
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.1, 1.0, n)
    M = _bernoulli_normal(rng, k, n, density)
    Qd = np.diag(D) + M.T @ M / 50.0
    Ad = _bernoulli_normal(rng, m, n, density)
    c = rng.standard_normal(n)
    A = sp.csr_matrix(Ad)
    b = _feasible_rhs(rng, A, n, m_eq)
    Qr, Qc, Qv = _csr_arrays(sp.csr_matrix(Qd))
    Ar, Ac, Av = _csr_arrays(A)
    return QPInstance(n, m, m_eq, Qr, Qc, Qv, Ar, Ac, Av, c, b,
                      name=f"dense_small(n={n},m={m},seed={seed})")


def _sym_dd_Q(rng, n: int, partners: int, std: float = 0.1) -> sp.csr_matrix:
    """diag(U[0.5,2]) + S, S mirrored random pattern, made diagonally dominant."""
    rows = np.repeat(np.arange(n, dtype=np.int64), partners)
    # j = i + U{1..n-1} mod n is uniform over j != i
    cols = (rows + rng.integers(1, n, size=rows.size)) % n
    vals = rng.normal(0.0, std, size=rows.size)
    S = sp.coo_matrix((np.concatenate([vals, vals]),
                       (np.concatenate([rows, cols]), np.concatenate([cols, rows]))),
                      shape=(n, n)).tocsr()
    S.sum_duplicates()
    u = rng.uniform(0.5, 2.0, n)
    absrow = np.asarray(abs(S).sum(axis=1)).ravel()
    return (S + sp.diags(u + absrow)).tocsr()


def _distinct_columns(rng, m: int, d: int, draw) -> np.ndarray:
    """m x d column indices, distinct within each row; duplicates are redrawn."""
    cols = draw(m * d).reshape(m, d)
    while True:
        cols.sort(axis=1)
        dup = np.zeros((m, d), dtype=bool)
        dup[:, 1:] = cols[:, 1:] == cols[:, :-1]
        bad_rows = np.nonzero(dup.any(axis=1))[0]
        if bad_rows.size == 0:
            return cols
        sub = cols[bad_rows]
        subdup = dup[bad_rows]
        sub[subdup] = draw(int(subdup.sum()))
        cols[bad_rows] = sub


def _row_csr(m: int, n: int, cols: np.ndarray, vals: np.ndarray) -> sp.csr_matrix:
    d = cols.shape[1]
    rowptr = np.arange(0, (m + 1) * d, d, dtype=np.int64)
    return sp.csr_matrix((vals.ravel(), cols.ravel(), rowptr), shape=(m, n))


def sparse_dd(seed: int = 0, n: int = 1_000_000, m: int = 500_000, q_partners: int = 4,
              a_row_nnz: int = 10, m_eq: int = 0) -> QPInstance:
    """The large sparse instance (Q diagonally dominant, A uniform columns)."""
    rng = np.random.default_rng(seed)
    Q = _sym_dd_Q(rng, n, q_partners)
    d = min(a_row_nnz, n)
    cols = _distinct_columns(rng, m, d, lambda k: rng.integers(0, n, size=k))
    A = _row_csr(m, n, cols, rng.standard_normal((m, d)))
    c = rng.standard_normal(n)
    b = _feasible_rhs(rng, A, n, m_eq)
    Qr, Qc, Qv = _csr_arrays(Q)
    Ar, Ac, Av = _csr_arrays(A)
    return QPInstance(n, m, m_eq, Qr, Qc, Qv, Ar, Ac, Av, c, b,
                      name=f"sparse_dd(n={n},m={m},seed={seed})")


def zipf_dd(seed: int = 0, n: int = 10_000_000, m: int = 5_000_000, s: float = 1.1,
            a_row_nnz: int = 8, m_eq: int = 0) -> QPInstance:
    """The largest instance: power-law (Zipf s) column popularity in A."""
    rng = np.random.default_rng(seed)
    Q = _sym_dd_Q(rng, n, 2) if n > 2 else sp.identity(n, format="csr")
    # a third partner for half of the rows gives ~5 nnz/row on average
    extra = rng.random(n) < 0.5
    if n > 2 and extra.any():
        rows = np.nonzero(extra)[0]
        cols = (rows + rng.integers(1, n, size=rows.size)) % n
        vals = rng.normal(0.0, 0.1, size=rows.size)
        E = sp.coo_matrix((np.concatenate([vals, vals]),
                           (np.concatenate([rows, cols]), np.concatenate([cols, rows]))),
                          shape=(n, n)).tocsr()
        E.sum_duplicates()
        Q = (Q + E + sp.diags(np.asarray(abs(E).sum(axis=1)).ravel())).tocsr()
    ranks = np.arange(1, n + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-s))
    cdf /= cdf[-1]
    perm = rng.permutation(n)
    d = min(a_row_nnz, n)

    def draw(k):
        r = np.searchsorted(cdf, rng.random(k), side="right")
        return perm[np.minimum(r, n - 1)]

    cols = _distinct_columns(rng, m, d, draw)
    A = _row_csr(m, n, cols, rng.standard_normal((m, d)))
    c = rng.standard_normal(n)
    b = _feasible_rhs(rng, A, n, m_eq)
    Qr, Qc, Qv = _csr_arrays(Q)
    Ar, Ac, Av = _csr_arrays(A)
    return QPInstance(n, m, m_eq, Qr, Qc, Qv, Ar, Ac, Av, c, b,
                      name=f"zipf_dd(n={n},m={m},seed={seed})")


def box_diag(seed: int = 0, n: int = 50) -> QPInstance:
    """Diagonal Q with the box l <= x <= u written as rows [I; -I] (closed form)."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.5, 2.0, n)
    c = rng.standard_normal(n) * 2.0
    lo = -rng.uniform(0.1, 1.0, n)
    hi = rng.uniform(0.1, 1.0, n)
    A = sp.vstack([sp.identity(n), -sp.identity(n)]).tocsr()
    b = np.concatenate([hi, -lo])
    Qr, Qc, Qv = _csr_arrays(sp.diags(q))
    Ar, Ac, Av = _csr_arrays(A)
    return QPInstance(n, 2 * n, 0, Qr, Qc, Qv, Ar, Ac, Av, c, b,
                      name=f"box_diag(n={n},seed={seed})", meta={"q": q, "lo": lo, "hi": hi})


def from_dense(Qd: np.ndarray, Ad: np.ndarray, c: np.ndarray, b: np.ndarray,
               m_eq: int = 0, name: str = "dense") -> QPInstance:
    """Wrap dense arrays as a CSR instance (explicit zeros dropped)."""
    Qr, Qc, Qv = _csr_arrays(sp.csr_matrix(Qd))
    A = sp.csr_matrix(Ad) if Ad.size else sp.csr_matrix((Ad.shape[0], Qd.shape[0]))
    Ar, Ac, Av = _csr_arrays(A)
    return QPInstance(Qd.shape[0], Ad.shape[0], m_eq, Qr, Qc, Qv, Ar, Ac, Av,
                      np.asarray(c, np.float64), np.asarray(b, np.float64), name=name)


# ---------------------------------------------------------------- low rank
@dataclass
class LowRankQP:
    """min 1/2 x'(F F' + diag(qd))x + c'x s.t. A x <= b (first m_eq rows =).

    F is n x k, row-major.  ``to_instance`` writes Q out explicitly (for the
    CPU oracle and the single-QP solver)."""

    n: int
    m: int
    m_eq: int
    k: int
    F: np.ndarray  # float64 [n, k]
    qd: np.ndarray  # float64 [n]
    A_rowptr: np.ndarray
    A_col: np.ndarray
    A_val: np.ndarray
    c: np.ndarray
    b: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)
    lo: np.ndarray | None = None  # variable bounds (+-inf where absent); None: none
    hi: np.ndarray | None = None

    def to_instance(self) -> QPInstance:
        Qd = self.F @ self.F.T + np.diag(self.qd)
        Qr, Qc, Qv = _csr_arrays(sp.csr_matrix(Qd))
        return QPInstance(self.n, self.m, self.m_eq, Qr, Qc, Qv, self.A_rowptr, self.A_col,
                          self.A_val, self.c, self.b, name=self.name, meta=dict(self.meta),
                          lo=self.lo, hi=self.hi)


def _portfolio_rows(n: int, sector: np.ndarray, s: int, bounds: bool = False):
    """A = [budget 1'; -I; sector indicator rows], b = [1; 0; 1.5 |S_j| / n].

    ``bounds``: the long-only rows -x <= 0 are left out (they become the
    variable bounds x >= 0): A = [budget 1'; sector rows]."""
    rows = [np.zeros(n, np.int64), 1 + sector]
    cols = [np.arange(n), np.arange(n)]
    vals = [np.ones(n), np.ones(n)]
    m = 1 + s
    if not bounds:
        rows = [rows[0], np.arange(1, n + 1), 1 + n + sector]
        cols = [cols[0], np.arange(n), np.arange(n)]
        vals = [vals[0], -np.ones(n), np.ones(n)]
        m = 1 + n + s
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m, n))
    A.sort_indices()
    size = np.bincount(sector, minlength=s).astype(np.float64)
    b = np.concatenate([[1.0]] + ([] if bounds else [np.zeros(n)]) + [1.5 * size / n])
    return A, b


def _low_rank_qp(F, qd, mu, sector, s, name, meta, bounds: bool = False) -> LowRankQP:
    n, k = F.shape
    A, b = _portfolio_rows(n, sector, s, bounds)
    Ar, Ac, Av = _csr_arrays(A)
    lo, hi = (np.zeros(n), np.full(n, np.inf)) if bounds else (None, None)
    return LowRankQP(n, A.shape[0], 1, k, np.ascontiguousarray(F, np.float64),
                     np.asarray(qd, np.float64), Ar, Ac, Av, -np.asarray(mu, np.float64), b,
                     name=name + (" bounds" if bounds else ""), meta=meta, lo=lo, hi=hi)


def portfolio(seed: int, index: int, n_lo: int = 20, n_hi: int = 400,
              bounds: bool = False) -> LowRankQP:
    """Instance ``index`` of ``portfolio_batch`` (its own substream).

    ``bounds``: the same problem with long-only written as the variable
    bounds x >= 0 instead of n rows of A (Section 4 solves it with BB
    projected-gradient x-steps)."""
    rng = np.random.default_rng([seed, index])
    n = int(rng.integers(n_lo, n_hi + 1))
    k = max(n // 10, 1)
    s = int(rng.integers(5, 21))
    F = rng.normal(0.0, np.sqrt(1.0 / k), size=(n, k))
    qd = rng.uniform(0.01, 0.1, n)
    mu = rng.normal(0.05, 0.02, n)
    sector = rng.integers(0, s, n)
    return _low_rank_qp(F, qd, mu, sector, s, f"portfolio(seed={seed},i={index},n={n})",
                        {"sectors": s}, bounds)


def portfolio_batch(seed: int = 0, count: int = 4096, n_lo: int = 20,
                    n_hi: int = 400, bounds: bool = False) -> list:
    return [portfolio(seed, i, n_lo, n_hi, bounds) for i in range(count)]


def portfolio_family(base_seed: int = 0, seeds=range(1, 21), n: int = 2000, k: int = 50,
                     sectors: int = 30, bounds: bool = False) -> list:
    """Instances of the parametric family: one per seed in ``seeds``."""
    base = np.random.default_rng([base_seed, 0])
    F0 = base.normal(0.0, np.sqrt(1.0 / k), size=(n, k))
    qd = base.uniform(0.01, 0.1, n)
    sector = base.integers(0, sectors, n)
    out = []
    for sd in seeds:
        rng = np.random.default_rng([base_seed, 1, int(sd)])
        mu = rng.normal(0.05, 0.02, n)
        F = F0 + 0.1 * np.sqrt(1.0 / k) * rng.standard_normal((n, k))
        out.append(_low_rank_qp(F, qd, mu, sector, sectors,
                                f"portfolio_family(base={base_seed},seed={sd})",
                                {"sectors": sectors, "mu": mu, "seed": int(sd)}, bounds))
    return out


# Named configurations used by the bench and the parity tests.
def make(name: str, seed: int = 0) -> QPInstance:
    if name == "dense_small":
        return dense_small(seed)
    if name == "sparse_dd":
        return sparse_dd(seed)
    if name == "sparse_dd_small":
        return sparse_dd(seed, n=20_000, m=10_000)
    if name == "zipf_dd":
        return zipf_dd(seed)
    if name == "zipf_dd_small":
        return zipf_dd(seed, n=20_000, m=10_000)
    raise KeyError(name)
