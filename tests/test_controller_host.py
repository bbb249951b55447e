"""Host logic of the controller trainer (no GPU): how a solver trace becomes
(features, action deviation, score) transitions."""
import numpy as np
import pytest

from paper_2609_19557_gb300 import controller as CT


def _trace(rows):
    tr = np.zeros((len(rows), 24))
    for k, (rel, inner, rule, taken) in enumerate(rows):
        tr[k, 1] = rel
        tr[k, 2] = inner
        tr[k, CT.F0:CT.F0 + CT.NF] = np.arange(CT.NF) + 100 * k
        tr[k, CT.A_RULE:CT.A_RULE + 2] = rule
        tr[k, CT.A_TAKEN:CT.A_TAKEN + 2] = taken
    return tr


def test_transitions_scores_and_deviations():
    tr = _trace([(1e-1, 0, (0.5, 0.0), (0.7, -0.2)),
                 (1e-3, 90, (0.4, 0.1), (0.4, 0.1)),
                 (1e-2, 990, (0.3, 0.0), (0.3, 0.0))])
    out = CT.transitions(tr)
    assert len(out) == 2  # the last action's outcome is not in the trace
    f, a, sc = out[0]
    assert np.array_equal(f, np.arange(CT.NF))
    assert a == pytest.approx([0.2, -0.2])
    # two decades of residual bought with log10(10 + 90) = 2 decades of work
    assert sc == pytest.approx(2.0 / 2.0)
    f, a, sc = out[1]
    assert np.array_equal(a, [0.0, 0.0])
    assert sc == pytest.approx(-1.0 / 3.0)  # the residual rose one decade for log10(1000) = 3


def test_transitions_guard_zero_residual():
    out = CT.transitions(_trace([(1e-2, 0, (0, 0), (0, 0)), (0.0, 0, (0, 0), (0, 0))]))
    assert np.isfinite(out[0][2]) and out[0][2] > 0


@pytest.mark.parametrize("d", [
    [-1, -2, 3, -4, -5, -1, -1, 0],
    [1] * 6 + [-1] * 6,
    [-3] * 18 + [2] * 14,
    [5, 7, 9],
    [0, 0],
])
def test_sign_test_matches_binomial_test(d):
    """The paired evaluation's exact two-sided sign test equals the exact binomial
    test of the number of negative differences among the nonzero ones (p = 1/2)."""
    st = pytest.importorskip("scipy.stats")
    k, nn, p = CT.sign_test(d)
    dd = np.asarray(d)
    assert k == int((dd < 0).sum()) and nn == int((dd != 0).sum())
    want = st.binomtest(k, nn, 0.5).pvalue if nn else 1.0
    assert abs(p - want) < 1e-12, (p, want)
