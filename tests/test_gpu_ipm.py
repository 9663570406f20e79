"""Stage 2 on the GPU (nmf_ipm, nmf_ipm_direction) against the oracle's
stage 2 (oracle_ipm_direction, oracle_ipm), through the C ABI.

* The Newton direction of eq. "eqn:equation" (Sec. 3.2: block Cholesky of
  R1, W = Cb P^-1, the Schur matrix and its dense Cholesky) with the
  Gauss-Newton blocks at random interior points, and with the full Hessian
  blocks near a stage-1 solution (where the method switches to them; at a
  random point the full system is indefinite): the same direction to 1e-9 of
  its largest entry (FP64 in both, different summation orders, a Schur
  matrix of moderate condition).
* The whole stage 2 (Alg. "alg:fast" after stage 1; Sec. 4's transition) on
  the square problems of the oracle's termination pins, where the printed
  method terminates: the GPU terminates too, after the oracle's number of
  Newton steps (+-2: the Armijo and switch decisions compare nearly equal
  numbers), at E(.;0) <= 1e-6 and the oracle's objective (1e-8).  A case
  counts only where the oracle's own run is robust to rounding: started from
  the stage-1 point perturbed by 1e-15 relative, it takes the same number of
  steps (some square starts, e.g. n = 20, seed 0, flip between terminating
  after 79 steps and drifting to the cap under such a perturbation).
* A config-1-shaped problem (n != m), where the printed method drifts along
  the scaling orbit: both reach the same Newton cap, at the same objective.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_08431_gb300 import StreamingNMF, build
    build.build()
    return StreamingNMF


def _handle(S, M, X, Y, prec=0):
    n, m = M.shape
    h = S(n, X.shape[1], m, prec=prec, kkt_target=0.0)
    h.append_columns(np.asfortranarray(M if prec == 0 else M.astype(np.float32)))
    h.set_factors(X, Y)
    return h


@pytest.mark.parametrize("full", [0, 1])
@pytest.mark.parametrize("n,m,k,prec", [(30, 12, 3, 0), (41, 17, 4, 1), (64, 20, 2, 0)])
def test_direction_matches_the_oracle(n, m, k, prec, full):
    S = _lib()
    g = np.random.default_rng(n + m + k + full)
    M, _, _ = synth.paper_uniform(n, m, k, sigma=0.1, seed=n)
    X, Y = synth.init_factors(n, m, k, seed=n)
    if full:
        X, Y, _, _, _, _, _ = oracle.anls(M, X, Y, max_sweeps=300)
        X, Y = X + 1e-3, Y + 1e-3                               # interior, near a stage-1 point
    else:
        X, Y = X + 0.05, Y + 0.05                               # interior
    R = g.uniform(0.1, 1.0, size=(n, k))
    Sd = g.uniform(0.1, 1.0, size=(k, m))
    mu, rho = 0.05, 1e-6
    ref = oracle.ipm_direction(M, X, Y, R, Sd, mu, rho, full)
    assert ref[4] == oracle.OK
    with _handle(S, M, X, Y, prec) as h:
        got = h.ipm_direction(R, Sd, mu, rho, full)
    for a, b in zip(got, ref[:4]):
        assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b)), np.max(np.abs(a - b)) / np.max(np.abs(b))


def _stage1(M, k, seed, stol=1e-5):
    n, m = M.shape
    X, Y = synth.init_factors(n, m, k, seed=seed)
    X, Y, _, _, _, _, st = oracle.anls(M, X, Y, max_sweeps=50000, stol=stol)
    assert st == oracle.OK
    return X, Y


@pytest.mark.parametrize("n,k,seed", [(24, 2, 0), (20, 2, 1), (12, 2, 0)])
def test_stage2_terminates_like_the_oracle_on_square_problems(n, k, seed):
    S = _lib()
    M, _, _ = synth.paper_uniform(n, n, k, sigma=0.1, seed=seed)
    X, Y = _stage1(M, k, seed)
    Xo, Yo, so, _, st = oracle.ipm(M, X, Y, eps_tol=1e-6, max_newton=400)
    assert st == oracle.OK
    g = np.random.default_rng(5)
    Xp = X * (1 + 1e-15 * g.standard_normal(X.shape))
    Yp = Y * (1 + 1e-15 * g.standard_normal(Y.shape))
    _, _, sp, _, stp = oracle.ipm(M, Xp, Yp, eps_tol=1e-6, max_newton=400)
    assert stp == oracle.OK and sp["newton"] == so["newton"]          # a robust case
    with _handle(S, M, X, Y) as h:
        sg = h.ipm(eps_tol=1e-6, max_newton=400)
        Xg, Yg, _, _ = h.get_factors()
    print("n=%d seed=%d: Newton steps GPU %d oracle %d; f %.12e vs %.12e" % (n, seed, sg["newton"], so["newton"],
                                                                           sg["f"], so["f"]))
    assert sg["status"] == 0 and sg["E0"] <= 1e-6
    assert abs(sg["newton"] - so["newton"]) <= 2
    assert sg["f"] == pytest.approx(so["f"], rel=1e-8)
    assert oracle.objective(M, Xg, Yg) == pytest.approx(so["f"], rel=1e-8)
    np.testing.assert_allclose(Xg @ Yg, Xo @ Yo, rtol=0, atol=1e-6 * np.abs(M).max())


def test_stage2_drifts_to_the_cap_like_the_oracle_when_n_differs_from_m():
    S = _lib()
    M, _, _ = synth.pdf_like(40, 12, 3, noise=1e-3, seed=0)
    X, Y = _stage1(M, 3, 0, stol=1e-4)
    _, _, so, _, st = oracle.ipm(M, X, Y, eps_tol=1e-6, max_newton=30)
    assert st == oracle.NOTCONV
    with _handle(S, M, X, Y) as h:
        sg = h.ipm(eps_tol=1e-6, max_newton=30, allow_notconv=True)
    assert sg["status"] == 4 and sg["newton"] == so["newton"] == 30
    assert sg["f"] == pytest.approx(so["f"], rel=1e-6)
