"""The oracle's warm-started Lawson-Hanson (Sec. 2: the previous problem's
solution seeds the next) against the cold solver, brute force, and the
paper's claim that along a chain of neighbouring columns the warm start
saves most of the active-set work."""
import numpy as np
import pytest

import oracle
import synth
from tests._brute import brute_nnls


def _spd(k, g, cond=1e3):
    Q, _ = np.linalg.qr(g.normal(size=(k, k)))
    return Q @ np.diag(np.geomspace(1.0, 1.0 / cond, k)) @ Q.T


def test_zero_warm_start_is_the_cold_solver():
    g = np.random.default_rng(0)
    for k in (1, 3, 8, 16):
        for _ in range(20):
            G = _spd(k, g)
            b = g.normal(size=k)
            yc, mc, oc, sc = oracle.nnls(G, b)
            yw, mw, ow, chw, sw = oracle.nnls_warm(G, b, np.zeros(k))
            assert sc == sw == oracle.OK
            assert np.array_equal(yc, yw) and mc == mw and oc == ow


@pytest.mark.parametrize("k", [2, 3, 4, 6])
def test_any_warm_start_reaches_the_brute_force_optimum(k):
    g = np.random.default_rng(10 + k)
    for _ in range(40):
        G = _spd(k, g, cond=50.0)
        b = g.normal(size=k)
        y0 = np.maximum(g.normal(size=k), 0.0)          # a random support and values
        yw, mw, ow, chw, sw = oracle.nnls_warm(G, b, y0)
        yb = brute_nnls(G, b)
        assert sw == oracle.OK
        assert np.allclose(yw, yb, rtol=1e-9, atol=1e-12), (yw, yb)


def test_warm_start_at_the_solution_takes_no_step():
    g = np.random.default_rng(3)
    for k in (4, 8, 16):
        for _ in range(10):
            G = _spd(k, g)
            b = g.normal(size=k)
            yc, mc, oc, sc = oracle.nnls(G, b)
            yw, mw, ow, chw, sw = oracle.nnls_warm(G, b, yc)
            assert sw == oracle.OK and ow == 0 and chw == 0 and mw == mc
            assert np.allclose(yw, yc, rtol=1e-12, atol=1e-15)


def test_chain_warm_start_saves_most_of_the_work():
    """PDF-like data after 100 sweeps: every column of the Y half solved cold
    and chained (column j seeded by column j - 1's solution).  The solutions
    agree to rounding (they are unique) and the chain takes a small fraction
    of the cold solver's entering steps, as Sec. 2 argues for streaming data
    whose neighbouring columns share their active set."""
    n, m, k = 400, 200, 4
    M, _, _ = synth.pdf_like(n, m, k, noise=1e-3, relative=True, seed=1)
    X, Y = synth.init_factors(n, m, k, seed=1)
    X, Y, _, _, _, _, st = oracle.anls(M, X, Y, max_sweeps=100)
    G = X.T @ X
    B = X.T @ M
    cold_steps = warm_steps = 0
    prev = np.zeros(k)
    for j in range(m):
        yc, _, oc, sc = oracle.nnls(G, B[:, j])
        yw, _, ow, chw, sw = oracle.nnls_warm(G, B[:, j], prev)
        assert sc == sw == oracle.OK
        assert np.allclose(yw, yc, rtol=1e-10, atol=1e-14 * max(np.abs(yc).max(), 1.0))
        cold_steps += oc
        warm_steps += ow
        prev = yw
    assert cold_steps >= m                      # every cold solve enters at least one variable
    assert warm_steps <= 0.25 * cold_steps, (warm_steps, cold_steps)
