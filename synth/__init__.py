"""Seeded synthetic inputs for the streaming-NMF workloads.

This module only draws numbers: it holds none of the factorisation's
arithmetic, so both the CPU oracle and the CUDA path may consume it.

Workloads (the paper's data sets are not available, so these stand in):

* ``pdf_like`` -- streaming "pair distribution function" data in the spirit of
  the AgMOR experiment of Sec. 5.2: each of the k true components X0[:, c] is a
  sum of 3-6 Gaussian peaks on a uniform distance grid (centre U[0, n), width
  U[2, 10] samples, height U[0.2, 1]); the phase fractions Y0[c, t] are smooth
  sigmoidal transitions in time that are nonnegative and sum to one per
  column (a sequential A -> B -> C ... reaction), so neighbouring time columns
  have nearly identical active sets (the continuity assumed in Sec. 1).
  M = X0 Y0 + N(0, sigma^2), with sigma absolute or relative to rms(X0 Y0).
* ``paper_uniform`` -- the synthetic recipe of Sec. 5.4: X, Y ~ U[0, 1],
  M = X Y + N(0, 0.1^2), negative entries set to zero.
* ``init_factors`` -- U[0, 1] starting factors (Alg. "alg:fast" leaves the
  initial point to the user).
* ``batch_problem_shapes`` -- uneven (n, m, k) draws for the batched workload.

M is rounded to float32 values and returned as float64, so an FP32 copy and
an FP64 copy of M hold exactly the same numbers and every precision mode
solves the same problem.
"""
from __future__ import annotations

import numpy as np

__all__ = ["pdf_like", "paper_uniform", "init_factors", "near_truth_factors",
           "batch_problem_shapes", "rng"]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed`` (every draw in this module goes through it)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _round_f32(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def pdf_like(n: int, m: int, k: int, noise: float = 1e-3, relative: bool = False,
             seed: int = 0, peaks: tuple[int, int] = (3, 6)):
    """PDF-like streaming data.

    Returns ``(M, X0, Y0)``: M is n x m (float64 holding float32 values, to be
    stored column-major), X0 is n x k, Y0 is k x m.
    """
    g = rng(seed)
    r = np.arange(n, dtype=np.float64)
    X0 = np.zeros((n, k))
    for c in range(k):
        npk = int(g.integers(peaks[0], peaks[1] + 1))
        centres = g.uniform(0.0, n, size=npk)
        widths = g.uniform(2.0, 10.0, size=npk)
        heights = g.uniform(0.2, 1.0, size=npk)
        for mu, w, h in zip(centres, widths, heights):
            X0[:, c] += h * np.exp(-0.5 * ((r - mu) / w) ** 2)
    # Sequential phase fractions: S_0 = 1 >= S_1(t) >= ... >= S_{k-1}(t) >= S_k = 0,
    # Y0[c] = S_c - S_{c+1}; equal logistic widths keep every difference >= 0.
    t = np.arange(m, dtype=np.float64)
    if k > 1:
        taus = np.sort(g.uniform(0.1 * m, 0.9 * m, size=k - 1))
        width = max(1.0, m / (4.0 * k)) * g.uniform(0.5, 1.5)
    S = np.ones((k + 1, m))
    S[k] = 0.0
    for c in range(1, k):          # S_c(t): fraction past the c-th transition
        S[c] = 1.0 / (1.0 + np.exp(-(t - taus[c - 1]) / width))
    Y0 = S[:-1] - S[1:]
    Y0 = np.maximum(Y0, 0.0)
    clean = X0 @ Y0
    sigma = noise * (np.sqrt(np.mean(clean ** 2)) if relative else 1.0)
    M = clean + g.normal(0.0, sigma, size=(n, m)) if sigma > 0 else clean.copy()
    return _round_f32(M), X0, Y0


def paper_uniform(n: int, m: int, k: int, sigma: float = 0.1, seed: int = 0):
    """Sec. 5.4 recipe: X, Y ~ U[0,1]; M = XY + N(0, sigma^2); negatives -> 0."""
    g = rng(seed)
    X0 = g.uniform(0.0, 1.0, size=(n, k))
    Y0 = g.uniform(0.0, 1.0, size=(k, m))
    M = X0 @ Y0 + g.normal(0.0, sigma, size=(n, m))
    M[M < 0] = 0.0
    return _round_f32(M), X0, Y0


def init_factors(n: int, m: int, k: int, seed: int = 0):
    """U[0,1] starting point: X (n x k), Y (k x m), both float64."""
    g = rng(seed + 7919)
    return g.uniform(0.0, 1.0, size=(n, k)), g.uniform(0.0, 1.0, size=(k, m))


def near_truth_factors(X0, Y0, rel: float = 0.1, seed: int = 0):
    """A starting point near the generating factors: X0 with every entry
    scaled by U[1 - rel, 1 + rel], and Y0 as it is (both float64 copies)."""
    g = rng(seed + 104729)
    X = np.asarray(X0, dtype=np.float64) * g.uniform(1.0 - rel, 1.0 + rel, size=np.shape(X0))
    return X, np.array(Y0, dtype=np.float64)


def batch_problem_shapes(nprob: int, seed0: int = 1000, n_range=(500, 4000),
                         m_range=(100, 2000), k_range=(2, 8)):
    """Uneven shapes for the batched workload: problem p draws from seed0 + p."""
    out = []
    for p in range(nprob):
        g = rng(seed0 + p)
        n = int(g.integers(n_range[0], n_range[1] + 1))
        m = int(g.integers(m_range[0], m_range[1] + 1))
        k = int(g.integers(k_range[0], k_range[1] + 1))
        out.append((n, m, k, seed0 + p))
    return out
