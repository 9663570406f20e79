"""Pins of the oracle's Lawson-Hanson NNLS (problem "qp", Sec. 2).

Nothing here re-runs the oracle's own formula: the checks are hand-worked
cases, exhaustive search over passive sets, the k = 1 closed form, the
unconstrained least-squares solution when it is interior, and the KKT
conditions of the subproblem.
"""
import os

import numpy as np
import pytest

import oracle
from tests._brute import brute_nnls, read_golden

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_problem(rs, k, rows=None, shift=0.3):
    rows = rows or 3 * k + 2
    C = rs.uniform(0, 1, size=(rows, k))
    d = rs.uniform(0, 1, size=rows) - shift * rs.uniform(0, 1, size=rows) * 2
    return C.T @ C, C.T @ d, C, d


@pytest.mark.parametrize("case", [1, 2, 3, 4, 5])
def test_hand_cases(case):
    g = read_golden(os.path.join(GOLD, "nnls_hand.txt"))
    b = np.atleast_1d(g["c%d_b" % case])
    k = b.shape[0]
    G = g["c%d_G" % case].reshape(k, k)
    y, mask, it, st = oracle.nnls(G, b)
    assert st == oracle.OK
    np.testing.assert_allclose(y, g["c%d_y" % case], rtol=1e-14, atol=1e-15)
    assert mask == sum(1 << i for i in range(k) if g["c%d_y" % case][i] > 0)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_brute_force_all_passive_sets(k):
    rs = np.random.default_rng(100 + k)
    for trial in range(60):
        G, b, _, _ = _rand_problem(rs, k, shift=rs.uniform(0, 0.8))
        y, mask, it, st = oracle.nnls(G, b)
        assert st == oracle.OK
        yb = brute_nnls(G, b)
        np.testing.assert_allclose(y, yb, rtol=1e-9, atol=1e-11 * max(1.0, np.abs(yb).max()))


def test_k1_closed_form():
    rs = np.random.default_rng(7)
    for _ in range(200):
        x = rs.uniform(0, 2, size=9)
        d = rs.normal(size=9)
        y, _, _, st = oracle.nnls(np.array([[x @ x]]), np.array([x @ d]))
        assert st == oracle.OK
        assert y[0] == pytest.approx(max(0.0, (x @ d) / (x @ x)), rel=1e-14, abs=1e-300)


def test_interior_equals_lstsq():
    rs = np.random.default_rng(11)
    hits = 0
    for _ in range(100):
        k = int(rs.integers(2, 7))
        C = rs.uniform(0, 1, size=(20, k))
        ytrue = rs.uniform(0.5, 2, size=k)
        d = C @ ytrue + 0.01 * rs.normal(size=20)
        ls = np.linalg.lstsq(C, d, rcond=None)[0]
        if np.all(ls > 0):
            hits += 1
            y, mask, _, st = oracle.nnls(C.T @ C, C.T @ d)
            assert st == oracle.OK and mask == (1 << k) - 1
            np.testing.assert_allclose(y, ls, rtol=1e-9)
    assert hits > 50


def test_subproblem_kkt():
    """y >= 0, gradient >= 0 off the support, ~0 on it, y o grad = 0."""
    rs = np.random.default_rng(3)
    for _ in range(300):
        k = int(rs.integers(1, 11))
        G, b, _, _ = _rand_problem(rs, k, shift=rs.uniform(0, 1))
        y, mask, _, st = oracle.nnls(G, b)
        assert st == oracle.OK
        grad = G @ y - b
        scale = np.abs(b).max() + np.abs(G).max() * max(1.0, y.max())
        assert np.all(y >= 0)
        assert np.all(grad >= -1e-12 * scale)
        assert np.all(np.abs(grad[y > 0]) <= 1e-11 * scale)
        assert np.abs(y * grad).max() <= 1e-11 * scale * max(1.0, y.max())


def test_all_negative_rhs_gives_zero():
    rs = np.random.default_rng(5)
    for k in (1, 3, 8):
        C = rs.uniform(0, 1, size=(12, k))
        d = -rs.uniform(0, 1, size=12)           # C >= 0, d < 0  =>  C'd < 0
        y, mask, _, st = oracle.nnls(C.T @ C, C.T @ d)
        assert st == oracle.OK and mask == 0 and np.all(y == 0)


def test_rank_deficient_gram_is_blocked_not_broken():
    """Two identical columns of C: G is singular; the solve stays finite and
    the fitted vector C y equals the fit of the reduced problem."""
    rs = np.random.default_rng(9)
    for _ in range(50):
        c = rs.uniform(0, 1, size=(15, 3))
        C = np.column_stack([c, c[:, 1]])        # column 3 duplicates column 1
        d = c @ rs.uniform(0.2, 1.0, size=3) + 0.01 * rs.normal(size=15)
        y, _, _, st = oracle.nnls(C.T @ C, C.T @ d)
        assert st == oracle.OK and np.all(np.isfinite(y)) and np.all(y >= 0)
        yr = brute_nnls(c.T @ c, c.T @ d)
        np.testing.assert_allclose(C @ y, c @ yr, rtol=1e-8, atol=1e-10)


def test_scale_invariance():
    """C -> aC, d -> cd  gives  y -> (c/a) y (the tolerance is scale free)."""
    rs = np.random.default_rng(21)
    for _ in range(50):
        k = int(rs.integers(2, 8))
        G, b, C, d = _rand_problem(rs, k)
        y, m0, _, _ = oracle.nnls(G, b)
        for a, c in ((1e-3, 1e4), (1e5, 1e-2)):
            y2, m2, _, _ = oracle.nnls((a * C).T @ (a * C), (a * C).T @ (c * d))
            assert m2 == m0
            np.testing.assert_allclose(y2, (c / a) * y, rtol=1e-9, atol=1e-12 * (c / a) * max(1, y.max()))
