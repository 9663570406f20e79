"""Pins of the oracle's objective, gradients and KKT error (eq. "prob",
eq. "eqn:kkt", eq. "error" with the ANLS duals of Sec. 5.1).

Independent evidence: hand-worked 2x2 cases, central finite differences of
f for the gradients, exact factorizations (zero error), and scale
equivariance of the relative figure.
"""
import os

import numpy as np
import pytest

import oracle
from tests._brute import read_golden

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("case", ["A", "B"])
def test_hand_cases(case):
    g = read_golden(os.path.join(GOLD, "kkt_hand.txt"))
    X = g[case + "_X"].reshape(2, 1)
    Y = g[case + "_Y"].reshape(1, 2)
    M = g[case + "_M"].reshape(2, 2)
    f, gX, gY = oracle.grad(M, X, Y)
    assert f == pytest.approx(g[case + "_f"], rel=1e-15)
    np.testing.assert_allclose(gX.ravel(), g[case + "_graX"], rtol=1e-15)
    np.testing.assert_allclose(gY.ravel(), g[case + "_graY"], rtol=1e-15)
    kk = oracle.kkt(M, X, Y)
    assert kk["E_abs"] == pytest.approx(g[case + "_E"], rel=1e-14)
    assert kk["s_g"] == pytest.approx(g[case + "_sg"], rel=1e-14)
    assert kk["rel"] == pytest.approx(g[case + "_rel"], rel=1e-14)
    assert kk["f"] == pytest.approx(g[case + "_f"], rel=1e-15)


def _f(M, X, Y):
    return 0.5 * np.sum((X @ Y - M) ** 2)


def test_gradients_match_finite_differences():
    rs = np.random.default_rng(0)
    n, m, k = 7, 5, 3
    M = rs.uniform(0, 1, size=(n, m))
    X = rs.uniform(0, 1, size=(n, k))
    Y = rs.uniform(0, 1, size=(k, m))
    _, gX, gY = oracle.grad(M, X, Y)
    h = 1e-6
    for i in range(n):
        for a in range(k):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, a] += h
            Xm[i, a] -= h
            fd = (_f(M, Xp, Y) - _f(M, Xm, Y)) / (2 * h)
            assert gX[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for a in range(k):
        for j in range(m):
            Yp, Ym = Y.copy(), Y.copy()
            Yp[a, j] += h
            Ym[a, j] -= h
            fd = (_f(M, X, Yp) - _f(M, X, Ym)) / (2 * h)
            assert gY[a, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_objective_is_half_squared_frobenius():
    rs = np.random.default_rng(1)
    for n, m, k in ((1, 1, 1), (9, 4, 2), (30, 17, 5)):
        M = rs.normal(size=(n, m))
        X = rs.uniform(size=(n, k))
        Y = rs.uniform(size=(k, m))
        # numpy's own norm routine on an explicit residual
        assert oracle.objective(M, X, Y) == pytest.approx(0.5 * np.linalg.norm(X @ Y - M) ** 2, rel=1e-13)


def test_exact_factorization_has_zero_error():
    rs = np.random.default_rng(2)
    X = rs.integers(0, 4, size=(6, 2)).astype(float)
    Y = rs.integers(0, 4, size=(2, 5)).astype(float)
    M = X @ Y                                   # small integers: exact in FP64
    kk = oracle.kkt(M, X, Y)
    assert kk["f"] == 0.0 and kk["E_abs"] == 0.0 and kk["rel"] == 0.0


def test_relative_kkt_scale_equivariance():
    """M -> cM with X -> sqrt(c) X, Y -> sqrt(c) Y leaves the relative figure
    unchanged and scales E_abs by c^2 (complementarity) or c^1.5 (signs)."""
    rs = np.random.default_rng(4)
    M = rs.uniform(size=(12, 9))
    X = rs.uniform(size=(12, 3))
    Y = rs.uniform(size=(3, 9))
    base = oracle.kkt(M, X, Y)
    for c in (1e-4, 37.0, 1e6):
        sc = oracle.kkt(c * M, np.sqrt(c) * X, np.sqrt(c) * Y)
        assert sc["rel"] == pytest.approx(base["rel"], rel=1e-12)
        assert sc["neg"] == pytest.approx(base["neg"] * c ** 1.5, rel=1e-12)
        assert sc["comp"] == pytest.approx(base["comp"] * c ** 2, rel=1e-12)
        assert sc["f"] == pytest.approx(base["f"] * c ** 2, rel=1e-12)


def test_sign_and_complementarity_terms_are_separated():
    """A point with only negative gradients has comp = 0; a point with only
    positive gradients on the support has neg = 0 (cases built by hand)."""
    # X=0 column: graY = X'(XY-M) = 0 for that row; use case A and B of the fixture
    g = read_golden(os.path.join(GOLD, "kkt_hand.txt"))
    kA = oracle.kkt(g["A_M"].reshape(2, 2), g["A_X"].reshape(2, 1), g["A_Y"].reshape(1, 2))
    kB = oracle.kkt(g["B_M"].reshape(2, 2), g["B_X"].reshape(2, 1), g["B_Y"].reshape(1, 2))
    assert kA["comp"] == 0.0 and kA["neg"] > 0
    assert kB["neg"] == 0.0 and kB["comp"] > 0
