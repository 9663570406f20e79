"""Per-column parity measures shared by the GPU tests (numpy only).

Parity is judged column by column (Y, k x m) and row by row (X, n x k), not
through one norm of the whole factor, so that a few wrong small columns
cannot hide under the bar of a large problem.

* ``colmax_rel`` -- max over columns of ||a_j - b_j|| / max(||b_j||, floor *
  max_j ||b_j||): relative per column, and absolute (against the factor's
  largest column) for columns far smaller than the largest.
* ``subproblem_excess`` / ``excess_bound`` -- the objective of each column's
  subproblem (eq. "qp", Sec. 2), phi(y) = 1/2 y'Gy - b'y with the reference's
  FP64 G and b.  y* (the reference) minimises phi over y >= 0, so the excess
  phi(y) - phi(y*) >= 0 measures how far the tested solution is from optimal
  in the sense that matters for the objective, and it stays well defined where
  the subproblem is ill conditioned and the values themselves are not.
  If the tested y minimises a perturbed problem, with b + d (|d_a| <= w_a) and
  G + E, then phi(y) <= phi(y*) + sum_a w_a |y_a - y*_a| to first order:
  phi'(y) <= phi'(y*) because y minimises phi', and phi - phi' is linear in
  the perturbation.  ``excess_bound`` returns that first-order bound.
"""
import numpy as np

import oracle


def colmax_rel(a, b, axis=0, floor=1e-3):
    """axis=0: columns of k x m factors; axis=1: rows of n x k factors."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(a - b, axis=axis)
    nb = np.linalg.norm(b, axis=axis)
    top = max(float(nb.max()) if nb.size else 0.0, 1e-300)
    return float(np.max(d / np.maximum(nb, floor * top))) if nb.size else 0.0


def subproblem_excess(G, B, V, Vref):
    """phi(v_j) - phi(vref_j) for every column j of V (k x m), computed
    without cancellation: 1/2 D'GD + sum over the reference's active
    components of the reference gradient (>= 0 there) times v."""
    D = V - Vref
    g = G @ Vref - B
    quad = 0.5 * np.einsum("aj,ab,bj->j", D, G, D)
    lin = np.sum(np.where(Vref > 0, 0.0, np.maximum(g, 0.0)) * np.maximum(V, 0.0), axis=0)
    return quad + lin


def excess_bound(G, Cabs, V, Vref, u, kappa, eps=0.0, B=None):
    """First-order bound of the excess: sum_a w_a |v_a - vref_a| with
    w = u * Cabs + kappa * |G| (|v| + |vref|) + tol.  Cabs (k x m) holds
    sum_r |X_ra| |M_rj| (the magnitude the contraction's rounding scales
    with); kappa covers the solve's own rounding of G and of the solution;
    tol is the Lawson-Hanson entering tolerance of the pass, 10 k eps
    (max|b| + max_a G_aa max|v|) (a variable whose gradient is below it
    does not enter, which is the exact optimum for b moved by that much)."""
    k = G.shape[0]
    W = u * Cabs + kappa * (np.abs(G) @ (np.abs(V) + np.abs(Vref)))
    if eps and B is not None:
        vmax = np.maximum(np.abs(V).max(axis=0), np.abs(Vref).max(axis=0))
        tol = 10.0 * k * eps * (np.abs(B).max(axis=0) + np.diag(G).max() * vmax)
        W = W + tol[None, :]
    return np.sum(W * np.abs(V - Vref), axis=0)


def phi_ref(B, Vref):
    """phi at the reference minimiser, -1/2 b'y* (<= 0)."""
    return -0.5 * np.sum(B * Vref, axis=0)


def mask_bits(mask, k):
    """uint32 passive-set masks (one per column) -> k x len(mask) booleans."""
    m = np.asarray(mask).astype(np.uint64)
    return ((m[None, :] >> np.arange(k, dtype=np.uint64)[:, None]) & np.uint64(1)).astype(bool)


def masks_differ_only_at_small_values(V, Vref, mask, mask_ref, cap):
    """Passive sets may differ only at entries whose value, on the side where
    it is positive, is at most cap times its column's largest reference value
    (a component the pass's rounding can move across zero).  V, Vref: k x m
    (for X pass the transposes).  Returns (ok, differing entries, the largest
    value at a difference over its column scale)."""
    k = Vref.shape[0]
    diff = mask_bits(mask, k) != mask_bits(mask_ref, k)
    scale = np.maximum(np.abs(Vref).max(axis=0, keepdims=True), 1e-300)
    rel = np.maximum(np.abs(V), np.abs(Vref)) / scale
    worst = float(rel[diff].max()) if diff.any() else 0.0
    return worst <= cap, int(diff.sum()), worst


# Rounding units of each M pass: u(L) bounds the relative error of one
# contraction entry of length L against sum |x| |m| (products plus a sum of L
# terms in any order); kappa the column / row solve's own rounding; eps the
# pass's Lawson-Hanson tolerance constant.
PASS_UNITS = {
    # FP64 products and sums; FP64 solves
    "fp64": dict(u=lambda L: (L + 1) * 2.0 ** -53, kappa=2.0 ** -40, eps=2.0 ** -52),
    # compensated FP32 (double-float, ~44 significant bits); FP64 solves
    "df": dict(u=lambda L: 2.0 ** -44 + L * 2.0 ** -47, kappa=2.0 ** -40, eps=2.0 ** -44),
    # FP32 products and sums; FP64 solves
    "f32": dict(u=lambda L: 2.0 ** -24 + 2.0 * (L - 1) * 2.0 ** -24, kappa=2.0 ** -40, eps=2.0 ** -52),
    # split-BF16 products (2^-15, tests/test_split_bf16_bound.py), FP32 sums;
    # FP32 column solves (kappa, eps), FP64 row solves (kappa_x, eps_x)
    "tc16": dict(u=lambda L: 2.0 ** -15 + 2.0 * (L - 1) * 2.0 ** -24, kappa=2.0 ** -18, kappa_x=2.0 ** -40,
                 eps=2.0 ** -23, eps_x=2.0 ** -23),
}


def solve_columns(G, B):
    """The oracle's NNLS of every column of B: (solutions k x cols, masks)."""
    out = [oracle.nnls(G, B[:, j]) for j in range(B.shape[1])]
    return np.stack([o[0] for o in out], axis=1), np.array([o[1] for o in out], dtype=np.uint32)


def objective_ratios(M, X, Xg, Yg, kind, J=None, I=None):
    """Each half-sweep of one GPU sweep from (X, .) against the oracle's solve
    of the same subproblems: the Y half with the input X (columns J, all by
    default), the X half with the GPU's new Y (rows I).  Returns the largest
    objective excess over its first-order bound for each half, (ry, rx), and
    the references (Yref, ymask_ref, Xref n x k, xmask_ref)."""
    U = PASS_UNITS[kind]
    n, m = M.shape
    Ms = M if J is None else M[:, J]
    G = X.T @ X
    B = X.T @ Ms
    Yref, ymo = solve_columns(G, B)
    Ys = Yg if J is None else Yg[:, J]
    exc = subproblem_excess(G, B, Ys, Yref)
    bnd = excess_bound(G, np.abs(X).T @ np.abs(Ms), Ys, Yref, U["u"](n), U["kappa"], U["eps"], B) + \
        1e-12 * np.abs(phi_ref(B, Yref))
    ry = float(np.max(exc / np.maximum(bnd, 1e-300)))
    H = Yg @ Yg.T
    Mr = M if I is None else M[I, :]
    Pt = Yg @ Mr.T
    Xref, xmo = solve_columns(H, Pt)
    Xs = (Xg if I is None else Xg[I, :]).T
    exc = subproblem_excess(H, Pt, Xs, Xref)
    bnd = excess_bound(H, np.abs(Yg) @ np.abs(Mr).T, Xs, Xref, U["u"](m), U.get("kappa_x", U["kappa"]),
                       U.get("eps_x", U["eps"]), Pt) + 1e-12 * np.abs(phi_ref(Pt, Xref))
    rx = float(np.max(exc / np.maximum(bnd, 1e-300)))
    return ry, rx, (Yref, ymo, Xref.T, xmo)
