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

WORKLOAD_CODES = {"small": 0, "mid": 1, "large": 2, "batched": 3, "learned": 4, "clique": 5,
                  "softlabel": 11, "flow": 12, "svm": 13}


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
             a_per_row: int = 4, neg_frac: float = 0.3, eq_frac: float = 0.2, shift: float = None) -> dict:
    """n=200, m=100 nonconvex QP with box [0,1]; ~30% negative eigenvalues of Q."""
    rng = _rng(seed, WORKLOAD_CODES["small"])
    k = int(round(q_offdiag_per_row * n))
    r = rng.integers(0, n, size=k)
    cc = rng.integers(0, n, size=k)
    off = _sym_offdiag(n, r, cc, rng.standard_normal(k))
    if shift is not None:
        pass  # given by the caller (a batch shares one replica's quantile)
    elif n <= 3000:
        shift = _quantile_shift(off, neg_frac)
    else:
        # Large n: the quantile from an n = 3000 replica with the same density.
        g = _rng(seed + 7919, WORKLOAD_CODES["small"])
        kr = int(round(q_offdiag_per_row * 3000))
        rep = _sym_offdiag(3000, g.integers(0, 3000, size=kr), g.integers(0, 3000, size=kr), g.standard_normal(kr))
        shift = _quantile_shift(rep, neg_frac)
    Q = (off + shift * sp.identity(n, format="csr")).tocsr()
    A = _rows_with_lengths(rng, n, np.full(m, a_per_row))
    c = rng.standard_normal(n)
    x0 = rng.uniform(0.0, 1.0, size=n)
    l_c, u_c = _constraint_bounds(rng, A, x0, eq_frac)
    return _pack(Q, c, A, l_c, u_c, np.zeros(n), np.ones(n), x0, workload="small", seed=seed, shift=shift)


def mid_qp(seed: int = 0, n: int = 50_000, m: int = 25_000, q_mean: float = 8.0, a_mean: float = 6.0,
           max_row: int = 200, free_frac: float = 0.1, eq_frac: float = 0.3, neg_frac: float = 0.3,
           replica_n: int = 3000, shift: float = None) -> dict:
    """Power-law rows (max 200 nnz), 10% free variables, 30% equality rows."""
    rng = _rng(seed, WORKLOAD_CODES["mid"])

    def q_off(nn: int, g: np.random.Generator) -> sp.csr_matrix:
        # Each row draws ~q_mean/2 partners; mirroring doubles the symmetric row mean.
        cnt = _power_law_lengths(g, nn, q_mean / 2.0, 1, max_row)
        rows = np.repeat(np.arange(nn), cnt)
        cols = g.integers(0, nn, size=rows.size)
        return _sym_offdiag(nn, rows, cols, g.standard_normal(rows.size))

    off = q_off(n, rng)
    if shift is None:  # else given by the caller (many instances of one density share it)
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


def _sorted_distinct(v: np.ndarray) -> np.ndarray:
    """Sorted distinct values (what np.unique returns; sort + neighbour test is faster for large v)."""
    v = np.sort(v)
    return v[np.concatenate(([True], v[1:] != v[:-1]))] if v.size else v


def _sym_pattern_csr(n: int, i: np.ndarray, j: np.ndarray) -> sp.csr_matrix:
    """0/1 symmetric CSR with sorted rows from distinct pairs i < j sorted by
    (i, j), written directly (row r: its lower neighbours, then its upper ones)."""
    k = i.size
    cl = np.bincount(j, minlength=n)
    cu = np.bincount(i, minlength=n)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cl + cu, out=indptr[1:])
    indices = np.empty(2 * k, dtype=np.int32)
    order = np.argsort(j, kind="stable")  # lower entries by row j, columns i ascending
    jl, il = j[order], i[order]
    indices[indptr[jl] + np.arange(k) - (np.cumsum(cl) - cl)[jl]] = il
    indices[indptr[i] + cl[i] + np.arange(k) - (np.cumsum(cu) - cu)[i]] = j
    return sp.csr_matrix((np.ones(2 * k), indices, indptr), shape=(n, n))


def clique_qp(seed: int = 0, n: int = 60, p: float = 0.1) -> dict:
    """Motzkin-Straus QP on G(n, p): min -x'A_G x s.t. sum(x) = 1, x >= 0 (Q = -2 A_G)."""
    rng = _rng(seed, WORKLOAD_CODES["clique"])
    if n <= 2000:
        iu = np.triu_indices(n, 1)
        mask = rng.random(iu[0].size) < p
        r, cc = iu[0][mask], iu[1][mask]
    else:
        # Large graphs: a Binomial number of edges, then distinct uniform
        # pairs i < j (the same distribution as the pairwise draws above).
        npairs = n * (n - 1) // 2
        k = int(rng.binomial(npairs, p))
        keys = _sorted_distinct(rng.integers(0, npairs, size=int(k * 1.1) + 16))
        while keys.size < k:
            keys = _sorted_distinct(np.concatenate([keys, rng.integers(0, npairs, size=k - keys.size + 16)]))
        keys = np.sort(rng.permutation(keys)[:k])
        # Pair index -> (i, j), i < j, row-major over the upper triangle.
        i = (n - 2 - np.floor(np.sqrt(-8.0 * keys + 4.0 * n * (n - 1) - 7) / 2.0 - 0.5)).astype(np.int64)
        j = (keys + i + 1 - n * (n - 1) // 2 + (n - i) * ((n - i) - 1) // 2).astype(np.int64)
        AG = _sym_pattern_csr(n, i, j)
        return _pack(-2.0 * AG, np.zeros(n), sp.csr_matrix(np.ones((1, n))), np.ones(1), np.ones(1), np.zeros(n),
                     np.full(n, np.inf), np.full(n, 1.0 / n), workload="clique", seed=seed, graph=AG)
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
    """Instance by workload name ("small", "mid", "large", "clique", "tiny", "softlabel", "flow", "svm")."""
    fn = {"small": small_qp, "mid": mid_qp, "large": large_qp, "clique": clique_qp, "tiny": tiny_qp,
          "softlabel": softlabel_qp, "flow": flow_qp, "svm": svm_qp}[workload]
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


# ---------------------------------------------------------------------------
# The paper's three million-variable model families (Appendix "Million-variable
# benchmark construction", parameter distributions of Table
# tab:million-generation, one default_rng stream per scenario; the family
# codes r = 1, 2, 3 of the paper are 11, 12, 13 here so that the streams do
# not coincide with those of the other generators).  The
# paper gives the models and the parameter ranges; how the graph, anchors and
# reference flows are drawn from those parameters is this module's reading.
# These are new instances, not the paper's frozen ones.
# ---------------------------------------------------------------------------
def _sym_from_upper(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> sp.csr_matrix:
    """Symmetric matrix from upper-triangle entries (i < j), mirrored exactly."""
    U = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    U.sum_duplicates()
    M = (U + U.T).tocsr()
    M.sort_indices()
    return M


def softlabel_qp(seed: int = 101, n_target: int = 1_000_000) -> dict:
    """Soft-label graph clustering: min -sum_{ij in E} w~_ij sum_c x_ic x_jc + sum a_ic x_ic
    s.t. sum_c x_ic = 1, 0 <= x <= 1, (1-delta) N/K <= sum_i x_ic <= (1+delta) N/K."""
    rng = _rng(seed, WORKLOAD_CODES["softlabel"])
    K = int(rng.choice([3, 5, 8, 10]))
    rg = int(rng.integers(8, 25))
    p_same = rng.uniform(0.55, 0.90)
    s_cross = rng.uniform(0.08, 0.45)
    sig_w = rng.uniform(0.10, 0.50)
    f_anchor = rng.uniform(0.03, 0.20)
    a_str = rng.uniform(0.5, 2.0)
    noise = rng.uniform(0.01, 0.08)
    delta = rng.uniform(0.05, 0.25)
    N = n_target // K
    labels = rng.permutation(np.arange(N) % K)  # balanced planted labelling
    # Reading: every vertex draws rg / 2 partners, of its own class with
    # probability p_same, otherwise of another class; weights are log-normal,
    # cross-class ones scaled by s_cross.
    half = max(1, rg // 2)
    src = np.repeat(np.arange(N), half)
    same = rng.random(src.size) < p_same
    dst = np.empty(src.size, dtype=np.int64)
    members = [np.flatnonzero(labels == k) for k in range(K)]
    for k in range(K):
        own = labels[src] == k
        m1 = own & same
        dst[m1] = members[k][rng.integers(0, members[k].size, size=int(m1.sum()))]
        m2 = own & ~same
        others = np.flatnonzero(labels != k)
        dst[m2] = others[rng.integers(0, others.size, size=int(m2.sum()))]
    keep = src != dst
    src, dst = src[keep], dst[keep]
    w = np.exp(sig_w * rng.standard_normal(src.size)) * np.where(labels[src] == labels[dst], 1.0, s_cross)
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    U = sp.coo_matrix((w, (lo, hi)), shape=(N, N)).tocsr()
    U.sum_duplicates()
    deg = np.asarray((U + U.T).sum(axis=1)).ravel()
    Uc = U.tocoo()
    wt = Uc.data / np.sqrt(deg[Uc.row] * deg[Uc.col])  # normalised weight, symmetric by construction
    Wt = _sym_from_upper(N, Uc.row, Uc.col, wt)
    Q = (-sp.kron(Wt, sp.identity(K, format="csr"), format="csr")).tocsr()
    Q.sort_indices()
    a = noise * rng.standard_normal((N, K))
    anchors = np.flatnonzero(rng.random(N) < f_anchor)
    a[anchors, labels[anchors]] -= a_str
    n = N * K
    ri = np.concatenate([np.repeat(np.arange(N), K), N + np.tile(np.arange(K), N)])
    ci = np.concatenate([np.arange(n), np.arange(n)])
    A = sp.csr_matrix((np.ones(2 * n), (ri, ci)), shape=(N + K, n))
    A.sort_indices()
    cap_lo, cap_hi = (1 - delta) * N / K, (1 + delta) * N / K
    l_c = np.concatenate([np.ones(N), np.full(K, cap_lo)])
    u_c = np.concatenate([np.ones(N), np.full(K, cap_hi)])
    return _pack(Q, a.ravel(), A, l_c, u_c, np.zeros(n), np.ones(n), np.full(n, 1.0 / K), workload="softlabel",
                 seed=seed, K=K, delta=delta, labels=labels)


def flow_qp(seed: int = 101, n_target: int = 1_000_000) -> dict:
    """Concave-cost multistage flow: min sum_e c_e f_e - alpha c_e / u_e f_e^2
    s.t. B f = b, 0 <= f <= u, on L layers of width w with three carriers."""
    rng = _rng(seed, WORKLOAD_CODES["flow"])
    L = int(rng.choice([4, 6, 8, 12, 16]))
    alpha = rng.uniform(0.03, 0.24)
    c0 = rng.uniform(0.05, 0.30)
    rho = rng.uniform(1.05, 1.80)
    growth = rng.uniform(0.0, 0.12)
    base = 1.0 / (1.0 - 2.0 * alpha)
    ratio = rng.uniform(base + 0.25, base + 2.0)  # geometric carrier-cost ratio
    h_lo, h_hi = rng.uniform(0.30, 1.00), rng.uniform(1.20, 3.00)
    h = rng.uniform(h_lo, h_hi, size=3)  # carrier reference-flow levels
    w = max(1, int(round(n_target / (3 * (L - 1)))))
    tails, heads, cost, f0 = [], [], [], []
    for stage in range(L - 1):
        for k in range(3):
            perm = rng.permutation(w)
            tails.append(stage * w + np.arange(w))
            heads.append((stage + 1) * w + perm)
            cost.append(np.full(w, c0 * ratio ** k * (1.0 + growth) ** stage))
            # Reading: arc reference flows scatter +-50 % around the carrier level.
            f0.append(h[k] * rng.uniform(0.5, 1.5, size=w))
    tails, heads = np.concatenate(tails), np.concatenate(heads)
    c, f0 = np.concatenate(cost), np.concatenate(f0)
    u = rho * f0
    ne, nv = tails.size, w * L
    B = sp.csr_matrix((np.concatenate([-np.ones(ne), np.ones(ne)]),
                       (np.concatenate([tails, heads]), np.concatenate([np.arange(ne), np.arange(ne)]))),
                      shape=(nv, ne))
    B.sort_indices()
    b = B @ f0
    Q = sp.diags(-2.0 * alpha * c / u, format="csr")
    return _pack(Q, c, B, b, b.copy(), np.zeros(ne), u, f0, workload="flow", seed=seed, L=L, alpha=alpha)


def svm_qp(seed: int = 101, n_target: int = 1_000_000) -> dict:
    """Indefinite graph-kernel SVM: min 1/2 a'Y K_eta Y a - 1'a s.t. y'a = 0,
    0 <= a <= U_alpha, K_eta = (1 - eta) I + eta D^-1/2 W D^-1/2 on a symmetric
    k-nearest-neighbour graph with W_ij = |tanh(kappa z_i'z_j / d)|."""
    from scipy.spatial import cKDTree
    rng = _rng(seed, WORKLOAD_CODES["svm"])
    d = int(rng.choice([4, 8, 12, 16]))
    k = int(rng.choice([6, 8, 12, 16, 24]))
    chi = rng.uniform(0.75, 3.00)
    nu = rng.uniform(0.50, 1.25)
    kappa = rng.uniform(0.75, 3.00)
    eta = rng.uniform(0.60, 0.97)
    Ua = rng.uniform(0.25, 2.00)
    N = n_target
    y = rng.permutation(np.where(np.arange(N) < N // 2, 1.0, -1.0))
    z = nu * rng.standard_normal((N, d))
    z[:, 0] += chi * y
    z[:, 1:] += 0.15 * rng.standard_normal((N, d - 1))
    _, nb = cKDTree(z).query(z, k=k + 1)
    src = np.repeat(np.arange(N), k)
    dst = nb[:, 1:].ravel()
    keep = src != dst
    lo, hi = np.minimum(src[keep], dst[keep]), np.maximum(src[keep], dst[keep])
    pairs = np.unique(lo * N + hi)  # symmetric kNN graph (union)
    lo, hi = pairs // N, pairs % N
    wv = np.abs(np.tanh(kappa * np.einsum("ij,ij->i", z[lo], z[hi]) / d))
    W = _sym_from_upper(N, lo, hi, wv)
    deg = np.asarray(W.sum(axis=1)).ravel()
    deg[deg == 0] = 1.0
    sv = eta * wv / np.sqrt(deg[lo] * deg[hi]) * y[lo] * y[hi]  # entries of Y K_eta Y off the diagonal
    Q = (_sym_from_upper(N, lo, hi, sv) + (1.0 - eta) * sp.identity(N, format="csr")).tocsr()
    Q.sort_indices()
    A = sp.csr_matrix(y.reshape(1, N))
    return _pack(Q, -np.ones(N), A, np.zeros(1), np.zeros(1), np.zeros(N), np.full(N, Ua), np.zeros(N),
                 workload="svm", seed=seed, eta=eta, labels=y)


def batched_shift(seed: int = 0) -> float:
    """Diagonal shift shared by the small-generator problems of a batch: the
    30 % eigenvalue quantile of an n = 2000 replica of its off-diagonal density."""
    g = _rng(seed + 7919, WORKLOAD_CODES["batched"])
    rep = _sym_offdiag(2000, g.integers(0, 2000, size=4000), g.integers(0, 2000, size=4000), g.standard_normal(4000))
    return _quantile_shift(rep, 0.3)


def batched_set(seed: int = 0, count: int = 256, n_lo: int = 1000, n_hi: int = 100_000,
                n_median: float = 4000.0, sigma: float = 0.8, clique_p: float = 0.01, only=None,
                mix: str = "alternate", shift: float = None) -> list:
    """A batch of independent problems of uneven sizes: n ~ lognormal (median
    n_median, log-std sigma, clipped to [n_lo, n_hi]); even positions use the
    small generator at that size with m = n / 2, odd positions Motzkin-Straus
    QPs on G(n, clique_p) (mix = "alternate"), or the small generator at every
    position (mix = "small").  Each problem has its own seed, so `only`
    (positions) builds a subset identical to those positions of the whole
    batch."""
    rng = _rng(seed, WORKLOAD_CODES["batched"])
    # One diagonal shift for the whole batch (batched_shift; a caller that
    # builds the batch in pieces computes it once and passes it).
    if shift is None:
        shift = batched_shift(seed)
    ns = np.clip(np.exp(np.log(n_median) + sigma * rng.standard_normal(count)), n_lo, n_hi).astype(np.int64)
    out = []
    keep = set(range(count)) if only is None else set(int(k) for k in only)
    for k, n in enumerate(ns):
        if k not in keep:
            continue
        s = int(seed) * 100_003 + k
        if k % 2 == 0 or mix == "small":
            out.append(small_qp(s, n=int(n), m=int(n) // 2, shift=shift))
        else:
            out.append(clique_qp(s, n=int(n), p=clique_p))
    return out
