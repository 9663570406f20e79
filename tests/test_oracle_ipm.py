"""Pins of the oracle's stage 2 (Alg. "alg:int" / "alg:fast", Sec. 3-4).

* The primal-dual direction (eq. "eqn:equation", solved through the Schur
  complement of Sec. 3.2) equals a dense numpy solve of the full 4-block
  Newton system whose Hessian is built by torch autograd: the full Hessian of
  f for the exact system, and J'J (J = Jacobian of the residual XY - M) for
  the Gauss-Newton system.  Neither the blocks Q1, Q2, C nor the Schur algebra
  are re-typed here.
* Finite termination with E(.;0) <= eps_TOL (Theorem "thm:converge") and a
  monotone merit function inside every inner loop (proof of the theorem).
* The two-stage result reaches the same local minimum as a tightly converged
  ANLS run from the same start.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")


def _vec(X, Y):
    return np.concatenate([np.asarray(X).ravel(order="C"), np.asarray(Y).ravel(order="F")])


def _autograd_hessians(M, X, Y):
    n, k = X.shape
    m = Y.shape[1]
    Mt = torch.tensor(M, dtype=torch.float64)

    def unpack(v):
        Xv = v[: n * k].reshape(n, k)
        Yv = v[n * k:].reshape(m, k).T          # y = vec(Y) (columns stacked)
        return Xv, Yv

    def f(v):
        Xv, Yv = unpack(v)
        return 0.5 * ((Xv @ Yv - Mt) ** 2).sum()

    def resid(v):
        Xv, Yv = unpack(v)
        return (Xv @ Yv - Mt).reshape(-1)

    v0 = torch.tensor(_vec(X, Y), dtype=torch.float64)
    H = torch.autograd.functional.hessian(f, v0).numpy()
    J = torch.autograd.functional.jacobian(resid, v0).numpy()
    v1 = v0.clone().requires_grad_(True)
    grad = torch.autograd.grad(f(v1), v1)[0].numpy()
    return H, J.T @ J, grad


@pytest.mark.parametrize("full", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_direction_equals_dense_newton_solve(full, seed):
    rs = np.random.default_rng(seed)
    n, m, k = 5, 4, 2
    X = rs.uniform(0.2, 1, size=(n, k))
    Y = rs.uniform(0.2, 1, size=(k, m))
    # near a fit, so that the exact Hessian (with the residual term) is PD too
    M = X @ Y + 0.05 * rs.normal(size=(n, m))
    R = rs.uniform(0.1, 0.5, size=(n, k))
    S = rs.uniform(0.1, 0.5, size=(k, m))
    mu, rho = 0.05, 1e-3
    dX, dY, dR, dS, st = oracle.ipm_direction(M, X, Y, R, S, mu, rho, full)
    assert st == oracle.OK
    Hfull, HGN, grad = _autograd_hessians(M, X, Y)
    Hm = (Hfull if full else HGN) + rho * np.eye(Hfull.shape[0])
    v = _vec(X, Y)
    d = _vec(R, S)
    N = v.size
    K = np.block([[Hm, -np.eye(N)], [np.diag(d), np.diag(v)]])
    rhs = np.concatenate([d - grad, mu - d * v])
    sol = np.linalg.solve(K, rhs)
    np.testing.assert_allclose(_vec(dX, dY), sol[:N], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(_vec(dR, dS), sol[N:], rtol=1e-9, atol=1e-12)


def test_gauge_identity_behind_the_drift():
    """sum_i graX_ic X_ic = sum_j graY_cj Y_cj for every column c, so along the
    orbit (X D, D^-1 Y) the barrier merit changes at rate -mu (n - m): it is
    unbounded below when n != m (why the n != m runs drift)."""
    rs = np.random.default_rng(12)
    for n, m, k in ((9, 4, 2), (5, 11, 3)):
        M = rs.uniform(size=(n, m))
        X = rs.uniform(0.1, 1, size=(n, k))
        Y = rs.uniform(0.1, 1, size=(k, m))
        _, gX, gY = oracle.grad(M, X, Y)
        for c in range(k):
            a, b = np.sum(gX[:, c] * X[:, c]), np.sum(gY[c] * Y[c])
            assert a == pytest.approx(b, rel=1e-12, abs=1e-14)


def _stage1(M, k, seed, stol=1e-5):
    n, m = M.shape
    X, Y = synth.init_factors(n, m, k, seed=seed)
    X, Y, _, _, sw, tr, st = oracle.anls(M, X, Y, max_sweeps=50000, stol=stol, want_trace=True)
    assert st == oracle.OK
    return X, Y, tr[-1, 0]


# Square problems (n = m) make phi invariant along the scaling orbit, so the
# hypotheses of Theorem "thm:converge" can hold; these draws of the Sec. 5.4
# recipe terminate.
SQUARE = [(20, 2, 0), (20, 2, 1), (20, 2, 2), (12, 2, 0), (12, 2, 1)]


@pytest.mark.parametrize("n,k,seed", SQUARE)
def test_ipm_finite_termination_and_monotone_merit(n, k, seed):
    M, _, _ = synth.paper_uniform(n, n, k, sigma=0.1, seed=seed)
    X, Y, f1 = _stage1(M, k, seed)
    Xi, Yi, stats, trace, st = oracle.ipm(M, X, Y, eps_tol=1e-6, max_newton=400, trace_cap=400)
    assert st == oracle.OK
    assert stats["E0"] <= 1e-6
    assert np.all(Xi > 0) and np.all(Yi > 0)
    assert stats["armijo_failures"] == 0
    for o in np.unique(trace[:, 0]):
        seg = trace[trace[:, 0] == o]
        assert np.all(seg[:, 3] <= seg[:, 2] + 1e-12 * np.abs(seg[:, 2]).max())
        assert np.all(seg[:, 1] == seg[0, 1])        # mu fixed inside the inner loop
    mus = [trace[trace[:, 0] == o][0, 1] for o in np.unique(trace[:, 0])]
    assert all(b < a for a, b in zip(mus, mus[1:]))   # mu decreases outer to outer
    # stage 2 never ends above where stage 1 stopped
    assert stats["f"] <= f1 * (1 + 1e-9)
    # the returned point also passes the ANLS-dual KKT test (separate function)
    assert oracle.kkt(M, Xi, Yi)["E_abs"] < 1e-5


def test_armijo_steps_decrease_phi_even_when_the_cap_ends_the_run():
    """n != m (config-1 shape, smaller): every accepted step still satisfies
    eq. "eqn:armijo"; the run itself ends at the Newton cap (see the gauge
    identity above)."""
    M, _, _ = synth.pdf_like(40, 12, 3, noise=1e-3, seed=0)
    X, Y, _ = _stage1(M, 3, 0, stol=1e-4)
    _, _, stats, trace, st = oracle.ipm(M, X, Y, eps_tol=1e-6, max_newton=200, trace_cap=200)
    assert st == oracle.NOTCONV and stats["newton"] == 200
    assert np.all(trace[:, 3] <= trace[:, 2])


def test_two_stage_reaches_the_converged_anls_minimum():
    n, k, seed = 20, 2, 0
    M, _, _ = synth.paper_uniform(n, n, k, sigma=0.1, seed=seed)
    X, Y = synth.init_factors(n, n, k, seed=seed)
    Xt, Yt, stats, st = oracle.two_stage(M, X, Y, stol=1e-5, max_sweeps=50000, eps_tol=1e-6)
    assert st == oracle.OK and stats["E0"] <= 1e-6
    Xa, Ya, _, _, sw, tr, st2 = oracle.anls(M, X, Y, max_sweeps=100000, kkt_target=1e-11, want_trace=True)
    assert st2 == oracle.OK and tr[-1, 2] <= 1e-11
    assert stats["f"] == pytest.approx(tr[-1, 0], rel=1e-8)
    np.testing.assert_allclose(Xt @ Yt, Xa @ Ya, rtol=0, atol=1e-4 * np.abs(M).max())
