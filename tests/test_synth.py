"""The seeded generators: reproducible, the stated structure, FP32-exact M."""
import numpy as np

import synth


def test_pdf_like_structure_and_determinism():
    M, X0, Y0 = synth.pdf_like(300, 80, 4, noise=1e-3, relative=True, seed=3)
    M2, _, _ = synth.pdf_like(300, 80, 4, noise=1e-3, relative=True, seed=3)
    np.testing.assert_array_equal(M, M2)
    assert M.shape == (300, 80) and X0.shape == (300, 4) and Y0.shape == (4, 80)
    assert np.all(X0 >= 0) and np.all(Y0 >= 0)
    np.testing.assert_allclose(Y0.sum(axis=0), 1.0, rtol=1e-12)
    assert np.array_equal(M, M.astype(np.float32).astype(np.float64))   # FP32-exact
    # neighbouring time columns are close (streaming continuity)
    d = np.abs(np.diff(Y0, axis=1)).max()
    assert d < 0.2


def test_paper_uniform_recipe():
    M, X0, Y0 = synth.paper_uniform(50, 20, 3, sigma=0.1, seed=1)
    assert np.all(M >= 0)
    assert np.all((X0 >= 0) & (X0 <= 1)) and np.all((Y0 >= 0) & (Y0 <= 1))


def test_batch_shapes_in_range():
    shapes = synth.batch_problem_shapes(64)
    assert len(shapes) == 64
    for n, m, k, seed in shapes:
        assert 500 <= n <= 4000 and 100 <= m <= 2000 and 2 <= k <= 8
    assert shapes == synth.batch_problem_shapes(64)
