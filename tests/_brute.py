"""Independent checkers used by the oracle pins (numpy only, no oracle code).

``brute_nnls`` solves min 1/2 y'Gy - b'y, y >= 0 by enumerating every passive
set P: the minimiser is the least-squares solution on its own support, so the
answer is the feasible (z_P >= 0) subset solution of least objective.
"""
import itertools

import numpy as np


def brute_nnls(G, b):
    G = np.asarray(G, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    k = b.shape[0]
    best, best_y = 0.0, np.zeros(k)          # P = {} gives y = 0, objective 0
    for size in range(1, k + 1):
        for P in itertools.combinations(range(k), size):
            P = list(P)
            try:
                z = np.linalg.solve(G[np.ix_(P, P)], b[P])
            except np.linalg.LinAlgError:
                continue
            if np.any(z < 0):
                continue
            y = np.zeros(k)
            y[P] = z
            obj = 0.5 * y @ G @ y - b @ y
            if obj < best:
                best, best_y = obj, y
    return best_y


def read_golden(path):
    """Parse a ``key = value`` text fixture (``#`` starts a comment)."""
    out = {}
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split("=", 1))
            vals = [float(v) for v in val.replace(",", " ").split()]
            out[key] = vals[0] if len(vals) == 1 else np.array(vals)
    return out
