"""The oracle's normal-probability estimator (HDR with subset-simulation
shifts, driven by the oracle's elliptical slice sampler) against what fixes
it independently of its own code:

* closed forms of Z = P(A x <= b), x ~ N(0, I): a halfspace (Phi(b / |a|)),
  an interval in d = 1, a box (a product of one-dimensional probabilities),
  and the orthant of a correlated bivariate normal (1/4 + asin(r) / (2 pi),
  Sheppard's formula), each within four standard errors of the estimator;
* exact counts: with one level the estimate is plain Monte Carlo over the
  stage's start draws, recounted here draw by draw with the residual of the
  row-by-row dot products; the first HDR level's count likewise;
* the structure the method fixes: shifts strictly decreasing to 0, k =
  ceil(rho n) samples inside every level of stage 1 but the last.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def _tol(counts, n):
    """Four standard errors of log Z: sum of (1 - p) / (n p) over the levels,
    inflated by 3 for the correlation of the chains' samples."""
    p = np.asarray(counts, dtype=float) / n
    return 4.0 * math.sqrt(3.0 * float(np.sum((1.0 - p) / (n * p))))


def _brute_count(A, b, X, gamma):
    """Samples with a_i . x - b_i <= gamma for every row, one dot product at a time."""
    cnt = 0
    for x in X:
        worst = max(sum(A[i, j] * x[j] for j in range(A.shape[1])) - b[i]
                    for i in range(A.shape[0]))
        cnt += worst <= gamma
    return cnt


def test_single_level_is_plain_monte_carlo():
    A = np.array([[1.0, 0.5]])
    b = np.array([1.2])
    n = 600
    r = oracle.hdr(A, b, n, rho=0.5, n_between=4, seed=7)
    assert list(r["shifts"]) == [0.0]
    X = oracle.hdr_start(8, n, 2)          # stage 2 draws (seed + 1)
    want = _brute_count(A, b, X, 0.0)
    assert r["counts"][0] == want
    assert r["log_z"] == pytest.approx(math.log(want / n), abs=1e-15)
    X1 = oracle.hdr_start(7, n, 2)         # stage 1 draws
    assert r["counts_ss"][0] == _brute_count(A, b, X1, 0.0)
    # the estimate is within Monte Carlo error of Phi(b / |a|)
    z = _phi(1.2 / math.hypot(1.0, 0.5))
    assert abs(want / n - z) <= 4 * math.sqrt(z * (1 - z) / n)


def test_halfspace_closed_form():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(4)
    A = a[None, :]
    b = np.array([-3.0 * np.linalg.norm(a)])
    n = 2000
    r = oracle.hdr(A, b, n, rho=0.5, n_between=8, seed=11)
    want = math.log(_phi(-3.0))
    assert len(r["shifts"]) >= 8
    assert abs(r["log_z"] - want) <= _tol(r["counts"], n), (r["log_z"], want)
    assert abs(r["log_z_ss"] - want) <= _tol(r["counts_ss"], n)


def test_interval_d1_closed_form():
    A = np.array([[1.0], [-1.0]])
    b = np.array([3.5, -2.0])                       # 2 <= x <= 3.5
    n = 2000
    r = oracle.hdr(A, b, n, rho=0.5, n_between=8, seed=5)
    want = math.log(_phi(3.5) - _phi(2.0))
    assert abs(r["log_z"] - want) <= _tol(r["counts"], n), (r["log_z"], want)


def test_box_product_closed_form():
    d = 3
    A = np.vstack([np.eye(d), -np.eye(d)])
    b = np.concatenate([np.full(d, 2.5), np.full(d, -1.0)])   # 1 <= x_j <= 2.5
    n = 2000
    r = oracle.hdr(A, b, n, rho=0.5, n_between=8, seed=9)
    want = d * math.log(_phi(2.5) - _phi(1.0))
    assert abs(r["log_z"] - want) <= _tol(r["counts"], n), (r["log_z"], want)


def test_correlated_orthant_sheppard():
    """y = L x with L L^T = [[1, r], [r, 1]]: P(y_1 <= 0, y_2 <= 0) =
    1/4 + asin(r) / (2 pi)."""
    r_corr = -0.9
    L = np.linalg.cholesky(np.array([[1.0, r_corr], [r_corr, 1.0]]))
    n = 2000
    r = oracle.hdr(L, np.zeros(2), n, rho=0.5, n_between=8, seed=13)
    want = math.log(0.25 + math.asin(r_corr) / (2 * math.pi))
    assert len(r["shifts"]) >= 3
    assert abs(r["log_z"] - want) <= _tol(r["counts"], n), (r["log_z"], want)


def test_shift_structure_and_first_hdr_count():
    rng = np.random.default_rng(3)
    d, m, n = 5, 12, 400
    A = rng.standard_normal((m, d))
    b = 0.3 + 0.1 * rng.standard_normal(m)   # contains the origin: not empty
    rho = 0.3
    k = math.ceil(rho * n)
    s1, c1 = oracle.hdr_stage(A, b, n, rho, 6, 21)
    assert s1[-1] == 0.0 and np.all(s1[:-1] > 0.0)
    assert np.all(np.diff(s1) < 0.0)
    assert np.all(c1[:-1] == k) and c1[-1] >= k
    s2, c2 = oracle.hdr_stage(A, b, n, rho, 6, 22, shifts=s1)
    np.testing.assert_array_equal(s2, s1[:len(s2)])
    X = oracle.hdr_start(22, n, d)
    assert c2[0] == _brute_count(A, b, X, s1[0])


def test_rejects_bad_rho():
    with pytest.raises(ValueError):
        oracle.hdr_stage(np.eye(2), np.ones(2), 10, 0.99, 2, 0)
