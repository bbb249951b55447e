"""Structure of the generators for the paper's million-variable model families
(Appendix "Million-variable benchmark construction"): soft-label graph
clustering, concave-cost multistage flow and the indefinite graph-kernel SVM,
checked on small instances against what each model fixes."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2609_19557_gb300 import instances as I


def _symmetric_exact(M):
    T = M.T.tocsr()
    T.sort_indices()
    return (np.array_equal(M.indptr, T.indptr) and np.array_equal(M.indices, T.indices)
            and np.array_equal(M.data, T.data))


def _feasible(inst, x, tol=1e-9):
    ax = inst["A"] @ x
    return (np.all(ax >= inst["l_c"] - tol) and np.all(ax <= inst["u_c"] + tol)
            and np.all(x >= inst["l_x"] - tol) and np.all(x <= inst["u_x"] + tol))


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_softlabel_structure(seed):
    inst = I.softlabel_qp(seed, n_target=3000)
    Q, A, K, delta = inst["Q"], inst["A"], inst["K"], inst["delta"]
    assert K in (3, 5, 8, 10) and 0.05 <= delta <= 0.25
    N = 3000 // K
    n = N * K
    assert Q.shape == (n, n) and A.shape == (N + K, n)
    assert _symmetric_exact(Q)
    # Q = -W~ (x) I_K: no entry couples two different labels, nonpositive,
    # zero diagonal (no self-loops).
    Qc = Q.tocoo()
    assert np.all(Qc.row % K == Qc.col % K)
    assert np.all(Qc.data < 0) and np.all(Q.diagonal() == 0)
    # Normalised weights: |w~_ij| <= 1 and the degree-normalised matrix has
    # spectral radius <= 1 (D^-1/2 W D^-1/2 is similar to a stochastic matrix).
    Wt = -Q[0::K, :][:, 0::K]
    lam = np.linalg.eigvalsh(Wt.toarray())
    assert lam.max() <= 1 + 1e-12 and lam.min() >= -1 - 1e-12
    # Simplex rows (K ones each, equalities = 1) then K capacity rows.
    rl = np.diff(A.indptr)
    assert np.all(rl[:N] == K) and np.all(rl[N:] == N) and np.all(A.data == 1.0)
    assert np.all(inst["l_c"][:N] == 1) and np.all(inst["u_c"][:N] == 1)
    assert np.allclose(inst["l_c"][N:], (1 - delta) * N / K) and np.allclose(inst["u_c"][N:], (1 + delta) * N / K)
    # x0 = 1/K is feasible; the planted labelling is balanced and feasible too.
    assert _feasible(inst, inst["x0"])
    lab = inst["labels"]
    assert np.all(np.bincount(lab, minlength=K) == N // K + (np.arange(K) < N % K))
    xp = np.zeros(n)
    xp[np.arange(N) * K + lab] = 1.0
    assert _feasible(inst, xp)


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_flow_structure(seed):
    inst = I.flow_qp(seed, n_target=3000)
    Q, B, L, alpha = inst["Q"], inst["A"], inst["L"], inst["alpha"]
    assert L in (4, 6, 8, 12, 16) and 0.03 <= alpha <= 0.24
    ne = Q.shape[0]
    w = ne // (3 * (L - 1))
    assert ne == 3 * w * (L - 1) and B.shape == (w * L, ne)
    # Incidence matrix: every arc leaves one node and enters one node of the
    # next layer.
    Bc = B.tocsc()
    assert np.all(np.diff(Bc.indptr) == 2)
    assert np.all(np.sort(Bc.data.reshape(-1, 2), axis=1) == [-1.0, 1.0])
    tails = np.where(Bc.data[0::2] < 0, Bc.indices[0::2], Bc.indices[1::2])
    heads = np.where(Bc.data[0::2] > 0, Bc.indices[0::2], Bc.indices[1::2])
    assert np.all(heads // w == tails // w + 1)
    # Concave separable cost: Q diagonal, f -> c f - alpha c f^2 / u, still
    # increasing on [0, u] (derivative c (1 - 2 alpha f / u) > 0 as alpha < 1/2).
    assert Q.nnz == ne and np.all(Q.indices == np.arange(ne))
    c, u = inst["c"], inst["u_x"]
    assert np.allclose(Q.diagonal(), -2 * alpha * c / u)
    assert np.all(c * (1 - 2 * alpha) > 0)
    # Flow conservation with b = B f0 and 0 <= f0 <= u.
    assert np.array_equal(inst["l_c"], inst["u_c"])
    assert np.allclose(B @ inst["x0"], inst["l_c"])
    assert _feasible(inst, inst["x0"], tol=1e-9)
    # Node balances sum to zero (every arc counted once with each sign).
    assert abs(inst["l_c"].sum()) <= 1e-9 * np.abs(inst["l_c"]).sum()


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_svm_structure(seed):
    inst = I.svm_qp(seed, n_target=1500)
    Q, A, eta, y = inst["Q"], inst["A"], inst["eta"], inst["labels"]
    N = 1500
    assert 0.6 <= eta <= 0.97
    assert _symmetric_exact(Q)
    assert np.allclose(Q.diagonal(), 1 - eta)
    # Q = Y K_eta Y with K_eta = (1 - eta) I + eta S, S = D^-1/2 W D^-1/2:
    # spectrum of K_eta in [1 - 2 eta, 1]; indefinite (the nonconvexity).
    K = (Q.multiply(np.outer(y, y))).toarray()
    lam = np.linalg.eigvalsh(K)
    assert lam.max() <= 1 + 1e-10 and lam.min() >= 1 - 2 * eta - 1e-10
    assert lam.max() == pytest.approx(1.0, abs=1e-8)  # the Perron vector D^1/2 1 of S (W >= 0)
    # Same spectrum for Q (a similarity by the sign matrix Y).
    assert np.allclose(np.linalg.eigvalsh(Q.toarray()), lam, atol=1e-9)
    # One dense equality row y'alpha = 0, balanced labels, box [0, U].
    assert A.shape == (1, N) and np.array_equal(A.toarray().ravel(), y)
    assert y.sum() == 0 and inst["l_c"][0] == 0 and inst["u_c"][0] == 0
    assert np.all(inst["u_x"] == inst["u_x"][0]) and 0.25 <= inst["u_x"][0] <= 2.0
    assert _feasible(inst, inst["x0"])


def test_families_are_deterministic():
    for f in (I.softlabel_qp, I.flow_qp, I.svm_qp):
        a, b = f(7, n_target=1200), f(7, n_target=1200)
        assert (a["Q"] != b["Q"]).nnz == 0 and (a["A"] != b["A"]).nnz == 0
        assert np.array_equal(a["c"], b["c"]) and np.array_equal(a["u_c"], b["u_c"])


def test_clique_sparse_sampler():
    """Large Motzkin-Straus graphs are drawn edge-list first: simple symmetric
    graph, zero diagonal, edge count within 5 standard deviations of p n (n-1) / 2."""
    n, p = 6000, 0.01
    inst = I.clique_qp(3, n=n, p=p)
    G = inst["graph"]
    assert _symmetric_exact(G) and G.diagonal().max() == 0 and np.all(G.data == 1.0)
    e = G.nnz // 2
    mu = p * n * (n - 1) / 2
    assert abs(e - mu) <= 5 * np.sqrt(mu)
    assert (inst["Q"] != -2.0 * G).nnz == 0


def test_oracle_solves_flow_family(oracle):
    """The oracle reaches rel-KKT 1e-4 on a small multistage-flow instance and
    its own external KKT test accepts the point (the family is solvable by
    the method as generated)."""
    inst = I.flow_qp(101, n_target=1500)
    x, y, info = oracle.solve(inst, eps_abs=1e-4, eps_rel=1e-4, time_limit=60)
    assert info["status"] == 0
    assert oracle.kkt_pass(inst, x, y, 1e-4, 1e-4)


def test_batched_set_structure():
    """Sizes inside the clip range, even positions from the small generator
    with m = n/2, odd positions Motzkin-Straus (one simplex row, Q = -2 A_G),
    one diagonal shift for the whole small-generator half, deterministic."""
    B = I.batched_set(3, count=6, n_lo=1000, n_hi=1500, n_median=1200, sigma=0.5)
    B2 = I.batched_set(3, count=6, n_lo=1000, n_hi=1500, n_median=1200, sigma=0.5)
    shifts = set()
    for k, (b, b2) in enumerate(zip(B, B2)):
        n = b["Q"].shape[0]
        assert 1000 <= n <= 1500
        assert (b["Q"] != b2["Q"]).nnz == 0 and np.array_equal(b["c"], b2["c"])
        assert _symmetric_exact(b["Q"])
        if k % 2 == 0:
            assert b["workload"] == "small" and b["A"].shape == (n, n // 2)[::-1]
            shifts.add(b["shift"])
            assert _feasible(b, b["x0"], tol=1e-9)
        else:
            assert b["workload"] == "clique" and b["A"].shape == (1, n)
            assert np.all(b["Q"].diagonal() == 0) and np.all(b["Q"].data == -2.0)
    assert len(shifts) == 1
