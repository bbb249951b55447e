"""Seeded synthetic nonconvex QP instances shaped like the paper's workloads.

Every instance is the problem of Eq. (qp) in two-sided form,

    min  c'x + 1/2 x'Qx   s.t.  l_c <= A x <= u_c,   l_x <= x <= u_x,

with Q symmetric (both triangles stored) and indefinite.  A row with
l_c == u_c is an equality row.  The paper's own million-variable and CUTEst
instances are not available, so these generators stand in for them (Sec. 4.1,
Appendix B/C): sparse local quadratic coupling, sparse general constraints,
and a feasible reference point x0 around which the constraint bounds are
built.

This module only draws random problem data.  It contains none of the
solver's arithmetic and is shared by the CUDA path's tests, the oracle's
tests and the benchmark.  Randomness follows the paper's convention of one
NumPy ``default_rng`` stream per instance seeded by ``SeedSequence([s, r])``
(Appendix C), with r the workload code below.

Workloads (sizes n x m):
    "small"  : n=200, m=100, 4 nnz/row in A, ~5 nnz/row in Q, box [0,1],
               20% equality rows, ~30% negative eigenvalues of Q.
    "mid"    : n=50,000, m=25,000, power-law row lengths (max 200) with means
               8 (Q) and 6 (A), 10% free variables, 30% equality rows.
    "large"  : n=1,000,000, m=500,000, Q = tridiagonal band + ~2 random
               symmetric entries/row (~5M nnz, ~20% negative eigenvalues),
               A = 8 nnz/row (4M nnz), box [-1,1], all rows two-sided.
    "clique" : Motzkin-Straus max-clique QP  min -x'A_G x  s.t. 1'x = 1, x >= 0
               on an Erdos-Renyi graph G(n, p).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

WORKLOAD_CODES = {"small": 0, "mid": 1, "large": 2, "batched": 3, "learned": 4, "clique": 5}


def _rng(seed: int, code: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(code)]))


def _sym_offdiag(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> sp.csr_matrix:
    """Symmetric matrix with the given (row, col) entries mirrored; diagonal hits dropped."""
    keep = rows != cols
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    # Sum repeated pairs once, in the upper triangle, then mirror the summed
    # values, so that both triangles hold bit-identical entries.
    lo, hi = np.minimum(rows, cols), np.maximum(rows, cols)
    U = sp.coo_matrix((vals, (lo, hi)), shape=(n, n)).tocsr()
    U.sum_duplicates()
    M = (U + U.T).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def _distinct_cols(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    """k distinct column indices in [0, n)."""
    if k <= 0:
        return np.zeros(0, dtype=np.int64)
    if 4 * k >= n:
        return np.sort(rng.choice(n, size=k, replace=False))
    out = np.unique(rng.integers(0, n, size=k + 8))
    while out.size < k:
        out = np.unique(np.concatenate([out, rng.integers(0, n, size=k)]))
    return np.sort(rng.choice(out, size=k, replace=False))


def _rows_with_lengths(rng: np.random.Generator, n_cols: int, lengths: np.ndarray) -> sp.csr_matrix:
    """CSR matrix whose row i has lengths[i] distinct random columns, N(0,1) values."""
    m = lengths.size
    lengths = np.minimum(lengths, n_cols).astype(np.int64)
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=indptr[1:])
    nnz = int(indptr[-1])
    # Draw with replacement, then repair duplicates row by row (rare for short rows).
    cols = rng.integers(0, n_cols, size=nnz)
    row_of = np.repeat(np.arange(m), lengths)
    key = row_of * n_cols + cols
    order = np.argsort(key, kind="stable")
    dup = np.zeros(nnz, dtype=bool)
    ks = key[order]
    dup[order[1:]] = ks[1:] == ks[:-1]
    for i in np.unique(row_of[dup]):
        a, b = indptr[i], indptr[i + 1]
        cols[a:b] = _distinct_cols(rng, n_cols, int(b - a))
    vals = rng.standard_normal(nnz)
    M = sp.csr_matrix((vals, cols, indptr), shape=(m, n_cols))
    M.sort_indices()
    return M


def _power_law_lengths(rng: np.random.Generator, count: int, mean: float, lo: int, hi: int) -> np.ndarray:
    """Discrete power-law (Zipf-like) lengths on [lo, hi] whose mean is ~mean.

    P(k) ~ k^(-a) on lo..hi with the exponent a fitted by bisection so that the
    truncated distribution's mean equals ``mean``.
    """
    ks = np.arange(lo, hi + 1, dtype=np.float64)

    def mean_of(a: float) -> float:
        w = ks ** (-a)
        return float((w * ks).sum() / w.sum())

    a_lo, a_hi = 0.0, 20.0
    for _ in range(200):
        a_mid = 0.5 * (a_lo + a_hi)
        if mean_of(a_mid) > mean:
            a_lo = a_mid
        else:
            a_hi = a_mid
    w = ks ** (-0.5 * (a_lo + a_hi))
    return rng.choice(ks.astype(np.int64), size=count, p=w / w.sum())


def _quantile_shift(off: sp.csr_matrix, frac_negative: float) -> float:
    """Diagonal shift s such that a fraction ``frac_negative`` of eig(off + s I) is negative."""
    ev = np.linalg.eigvalsh(off.toarray())
    return -float(np.quantile(ev, frac_negative))


def _constraint_bounds(rng, A, x0, eq_frac):
    ax = A @ x0
    m = A.shape[0]
    lo = ax - rng.uniform(0.1, 1.0, size=m)
    hi = ax + rng.uniform(0.1, 1.0, size=m)
    n_eq = int(round(eq_frac * m))
    if n_eq:
        eq = rng.choice(m, size=n_eq, replace=False)
        lo[eq] = ax[eq]
        hi[eq] = ax[eq]
    return lo, hi


def _pack(Q, c, A, l_c, u_c, l_x, u_x, x0, **meta):
    Q = Q.tocsr()
    A = A.tocsr()
    Q.sort_indices()
    A.sort_indices()
    d = dict(Q=Q, c=np.ascontiguousarray(c, dtype=np.float64), A=A,
             l_c=np.ascontiguousarray(l_c, dtype=np.float64), u_c=np.ascontiguousarray(u_c, dtype=np.float64),
             l_x=np.ascontiguousarray(l_x, dtype=np.float64), u_x=np.ascontiguousarray(u_x, dtype=np.float64),
             x0=np.ascontiguousarray(x0, dtype=np.float64))
    d.update(meta)
    return d


def small_qp(seed: int = 0, n: int = 200, m: int = 100, q_offdiag_per_row: float = 2.0,
             a_per_row: int = 4, neg_frac: float = 0.3, eq_frac: float = 0.2) -> dict:
    """n=200, m=100 nonconvex QP with box [0,1]; ~30% negative eigenvalues of Q."""
    rng = _rng(seed, WORKLOAD_CODES["small"])
    k = int(round(q_offdiag_per_row * n))
    r = rng.integers(0, n, size=k)
    cc = rng.integers(0, n, size=k)
    off = _sym_offdiag(n, r, cc, rng.standard_normal(k))
    shift = _quantile_shift(off, neg_frac)
    Q = (off + shift * sp.identity(n, format="csr")).tocsr()
    A = _rows_with_lengths(rng, n, np.full(m, a_per_row))
    c = rng.standard_normal(n)
    x0 = rng.uniform(0.0, 1.0, size=n)
    l_c, u_c = _constraint_bounds(rng, A, x0, eq_frac)
    return _pack(Q, c, A, l_c, u_c, np.zeros(n), np.ones(n), x0, workload="small", seed=seed, shift=shift)


def mid_qp(seed: int = 0, n: int = 50_000, m: int = 25_000, q_mean: float = 8.0, a_mean: float = 6.0,
           max_row: int = 200, free_frac: float = 0.1, eq_frac: float = 0.3, neg_frac: float = 0.3,
           replica_n: int = 3000) -> dict:
    """Power-law rows (max 200 nnz), 10% free variables, 30% equality rows."""
    rng = _rng(seed, WORKLOAD_CODES["mid"])

    def q_off(nn: int, g: np.random.Generator) -> sp.csr_matrix:
        # Each row draws ~q_mean/2 partners; mirroring doubles the symmetric row mean.
        cnt = _power_law_lengths(g, nn, q_mean / 2.0, 1, max_row)
        rows = np.repeat(np.arange(nn), cnt)
        cols = g.integers(0, nn, size=rows.size)
        return _sym_offdiag(nn, rows, cols, g.standard_normal(rows.size))

    off = q_off(n, rng)
    rep = q_off(min(replica_n, n), _rng(seed + 7919, WORKLOAD_CODES["mid"]))
    shift = _quantile_shift(rep, neg_frac)
    Q = (off + shift * sp.identity(n, format="csr")).tocsr()
    lens = _power_law_lengths(rng, m, a_mean, 1, max_row)
    A = _rows_with_lengths(rng, n, lens)
    l_x, u_x = np.zeros(n), np.ones(n)
    n_free = int(round(free_frac * n))
    free = rng.choice(n, size=n_free, replace=False)
    l_x[free], u_x[free] = -np.inf, np.inf
    # Keep the feasible set bounded along the free variables: n_free distinct
    # "pivot" rows each hold exactly one free variable (coefficient of magnitude
    # in [0.5, 1.5]) and no other free variable, so that every free variable is
    # confined by its pivot row's two-sided bounds given the boxed variables.
    is_free = np.zeros(n, dtype=bool)
    is_free[free] = True
    pivots = rng.choice(m, size=n_free, replace=False)
    Acoo = A.tocoo()
    drop = np.isin(Acoo.row, pivots) & is_free[Acoo.col]
    pr = pivots
    pc = rng.permutation(free)
    pv = rng.choice([-1.0, 1.0], size=n_free) * rng.uniform(0.5, 1.5, size=n_free)
    keep = ~drop
    rows = np.concatenate([Acoo.row[keep], pr])
    cols = np.concatenate([Acoo.col[keep], pc])
    vals = np.concatenate([Acoo.data[keep], pv])
    A = sp.coo_matrix((vals, (rows, cols)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    c = rng.standard_normal(n)
    x0 = rng.uniform(0.0, 1.0, size=n)
    x0[free] = rng.uniform(-1.0, 1.0, size=n_free)
    l_c, u_c = _constraint_bounds(rng, A, x0, eq_frac)
    return _pack(Q, c, A, l_c, u_c, l_x, u_x, x0, workload="mid", seed=seed, shift=shift)


def large_qp(seed: int = 0, n: int = 1_000_000, m: int = 500_000, a_per_row: int = 8,
             rand_per_row: float = 1.0, neg_frac: float = 0.2, replica_n: int = 4000) -> dict:
    """n=1e6, m=5e5: banded + random sparse indefinite Q, 8 nnz/row A, box [-1,1]."""
    rng = _rng(seed, WORKLOAD_CODES["large"])

    def q_off(nn: int, g: np.random.Generator) -> sp.csr_matrix:
        i = np.arange(nn - 1)
        band_v = g.standard_normal(nn - 1)
        k = int(round(rand_per_row * nn))
        rr = g.integers(0, nn, size=k)
        rc = g.integers(0, nn, size=k)
        return _sym_offdiag(nn, np.concatenate([i, rr]), np.concatenate([i + 1, rc]),
                            np.concatenate([band_v, g.standard_normal(k)]))

    off = q_off(n, rng)
    rep = q_off(min(replica_n, n), _rng(seed + 7919, WORKLOAD_CODES["large"]))
    shift = _quantile_shift(rep, neg_frac)
    Q = (off + shift * sp.identity(n, format="csr")).tocsr()
    A = _rows_with_lengths(rng, n, np.full(m, a_per_row))
    c = rng.standard_normal(n)
    x0 = rng.uniform(-1.0, 1.0, size=n)
    l_c, u_c = _constraint_bounds(rng, A, x0, 0.0)
    return _pack(Q, c, A, l_c, u_c, -np.ones(n), np.ones(n), x0, workload="large", seed=seed, shift=shift)


def clique_qp(seed: int = 0, n: int = 60, p: float = 0.1) -> dict:
    """Motzkin-Straus QP on G(n, p): min -x'A_G x s.t. sum(x) = 1, x >= 0 (Q = -2 A_G)."""
    rng = _rng(seed, WORKLOAD_CODES["clique"])
    iu = np.triu_indices(n, 1)
    mask = rng.random(iu[0].size) < p
    r, cc = iu[0][mask], iu[1][mask]
    G = sp.coo_matrix((np.ones(r.size), (r, cc)), shape=(n, n))
    AG = (G + G.T).tocsr()
    Q = (-2.0 * AG).tocsr()
    if Q.nnz == 0:
        Q = sp.csr_matrix((n, n))
    A = sp.csr_matrix(np.ones((1, n)))
    return _pack(Q, np.zeros(n), A, np.ones(1), np.ones(1), np.zeros(n), np.full(n, np.inf),
                 np.full(n, 1.0 / n), workload="clique", seed=seed, graph=AG)


def tiny_qp(seed: int, n: int = 4, m: int = 2, convex: bool = False, eq_rows: int = 0,
            dense_frac: float = 0.7) -> dict:
    """Tiny dense-ish QP for brute-force checks (n <= 10)."""
    rng = _rng(seed, 100 + n * 10 + m)
    M = rng.standard_normal((n, n)) * (rng.random((n, n)) < dense_frac)
    Q = 0.5 * (M + M.T)
    if convex:
        Q = Q @ Q.T + 0.5 * np.eye(n)
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < dense_frac)
    for i in range(m):
        if not A[i].any():
            A[i, rng.integers(0, n)] = 1.0
    c = rng.standard_normal(n)
    x0 = rng.uniform(0.0, 1.0, size=n)
    ax = A @ x0
    l_c = ax - rng.uniform(0.1, 1.0, size=m)
    u_c = ax + rng.uniform(0.1, 1.0, size=m)
    for i in range(min(eq_rows, m)):
        l_c[i] = u_c[i] = ax[i]
    return _pack(sp.csr_matrix(Q), c, sp.csr_matrix(A), l_c, u_c, np.zeros(n), np.ones(n), x0,
                 workload="tiny", seed=seed)


def make(workload: str, seed: int = 0, **kw) -> dict:
    """Instance by workload name ("small", "mid", "large", "clique", "tiny")."""
    fn = {"small": small_qp, "mid": mid_qp, "large": large_qp, "clique": clique_qp, "tiny": tiny_qp}[workload]
    return fn(seed=seed, **kw)


def primal_infeasible_qp(seed: int = 0, n: int = 40, m: int = 20) -> dict:
    """The small generator with one extra row 1'x_S >= 10 over 5 boxed variables
    (x in [0, 1]): the constraint set is empty."""
    inst = small_qp(seed, n=n, m=m)
    rng = _rng(seed, WORKLOAD_CODES["small"] + 100)
    cols = np.sort(rng.choice(n, size=5, replace=False))
    row = sp.csr_matrix((np.ones(5), (np.zeros(5, dtype=int), cols)), shape=(1, n))
    A = sp.vstack([inst["A"], row]).tocsr()
    A.sort_indices()
    l_c = np.append(inst["l_c"], 10.0)
    u_c = np.append(inst["u_c"], np.inf)
    return _pack(inst["Q"], inst["c"], A, l_c, u_c, inst["l_x"], inst["u_x"], inst["x0"], workload="primal_inf",
                 seed=seed, row_cols=cols)


def dual_infeasible_qp(seed: int = 0, n: int = 40, m: int = 20) -> dict:
    """The small generator with variable 0 made free, removed from every row
    and from Q's off-diagonal part, and Q_00 = -1: the objective is unbounded
    below along x_0."""
    inst = small_qp(seed, n=n, m=m)
    Q = inst["Q"].tolil()
    Q[0, :] = 0.0
    Q[:, 0] = 0.0
    Q[0, 0] = -1.0
    Q = Q.tocsr()
    Q.eliminate_zeros()
    A = inst["A"].tolil()
    A[:, 0] = 0.0
    A = A.tocsr()
    A.eliminate_zeros()
    l_x, u_x = inst["l_x"].copy(), inst["u_x"].copy()
    l_x[0], u_x[0] = -np.inf, np.inf
    x0 = inst["x0"].copy()
    x0[0] = 0.0
    l_c, u_c = inst["l_c"].copy(), inst["u_c"].copy()
    ax = A @ x0  # keep the rows feasible at x0 after removing column 0
    lo_gap, hi_gap = inst["A"] @ inst["x0"] - inst["l_c"], inst["u_c"] - inst["A"] @ inst["x0"]
    l_c, u_c = ax - lo_gap, ax + hi_gap
    return _pack(Q, inst["c"], A, l_c, u_c, l_x, u_x, x0, workload="dual_inf", seed=seed)
