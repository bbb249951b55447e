"""Anderson acceleration of the oracle (Sec. "Anderson acceleration"), pinned
to facts of the method outside the oracle: on an affine map u -> M u + b of
dimension d, Type-II Anderson with d + 1 stored iterates of the plain
iteration returns the fixed point (I - M)^{-1} b (it is then equivalent to
GMRES on (I - M) u = b); with one stored pair there is no step; end-to-end
solves with it on or off both reach the tolerance."""
import numpy as np
import pytest

from paper_2609_19557_gb300 import instances as I


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_affine_map_fixed_point(oracle, d):
    rng = np.random.default_rng(d)
    M = 0.5 * rng.normal(size=(d, d)) / np.sqrt(d)
    b = rng.normal(size=d)
    u = [rng.normal(size=d)]
    for _ in range(d):
        u.append(M @ u[-1] + b)
    U = np.array(u)
    G = U @ M.T + b
    got = oracle.anderson_step(U, G)
    want = np.linalg.solve(np.eye(d) - M, b)
    assert np.allclose(got, want, rtol=1e-8, atol=1e-8), (got, want)


def test_single_pair_gives_no_step(oracle):
    assert oracle.anderson_step(np.ones((1, 3)), np.zeros((1, 3))) is None


@pytest.mark.parametrize("seed", [0, 1])
def test_solves_with_and_without_anderson(oracle, seed):
    inst = I.small_qp(seed)
    for aa in (0, 1):
        x, y, info = oracle.solve(inst, eps_abs=1e-6, eps_rel=1e-6, time_limit=60, anderson=aa)
        assert info["status_name"] == "SOLVED"
        assert oracle.kkt_pass(inst, x, y, 1e-6, 1e-6)
