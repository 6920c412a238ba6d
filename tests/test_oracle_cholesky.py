"""Pins of the oracle's Cholesky factor (App. A needs Sigma = L L^T).

* A hand-computed 3 x 3 case: L chosen, S = L L^T multiplied out by hand.
* Reconstruction L L^T = S on random positive definite matrices, with L lower
  triangular and a positive diagonal.
* The library routine (numpy.linalg.cholesky) gives the same factor: the
  Cholesky factor with positive diagonal is unique.
* A matrix that is not positive definite is refused at the right row.
"""
import numpy as np
import pytest

import oracle


def test_hand_computed_3x3():
    # L = [[2, 0, 0], [1, 3, 0], [-1, 2, 4]]:
    # row 0: (4, 2, -2); row 1: (2, 1 + 9, -1 + 6); row 2: (-2, 5, 1 + 4 + 16)
    S = np.array([[4.0, 2.0, -2.0], [2.0, 10.0, 5.0], [-2.0, 5.0, 21.0]])
    L = oracle.cholesky(S)
    np.testing.assert_allclose(L, [[2.0, 0.0, 0.0], [1.0, 3.0, 0.0], [-1.0, 2.0, 4.0]],
                               rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 150])
def test_reconstruction_and_uniqueness(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    S = M @ M.T + n * np.eye(n)
    L = oracle.cholesky(S)
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) > 0.0)
    np.testing.assert_allclose(L @ L.T, S, rtol=0, atol=1e-12 * np.abs(S).max())
    np.testing.assert_allclose(L, np.linalg.cholesky(S), rtol=0, atol=1e-12 * np.abs(L).max())


def test_reads_only_the_lower_triangle():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((6, 6))
    S = M @ M.T + np.eye(6)
    junk = S.copy()
    junk[np.triu_indices(6, 1)] = 1e30
    np.testing.assert_array_equal(oracle.cholesky(junk), oracle.cholesky(S))


def test_not_positive_definite():
    S = np.array([[4.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])  # row 1 pivot: 1 - 1 = 0
    with pytest.raises(ValueError, match="row 1"):
        oracle.cholesky(S)
