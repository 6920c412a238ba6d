"""Pins of the oracle's Sec. 3.3 trimming (the reading: endpoints that are
constraint angles move inwards by eps, the glued point theta = 0 / 2 pi never
moves, a piece whose ends cross is dropped, and trimming applies to I_act
after the intersection).

* A hand-derived case: three infeasible arcs placed at chosen angles with the
  construction of the Fig. 1 worked example; trimming shortens the pieces by
  eps at their constraint ends, leaves 0 and 2 pi fixed, and drops the short
  piece once 2 eps exceeds its length.
* A theta-grid brute force of the trimmed set on tiny random instances: a
  theta belongs to it exactly when every angle within eps of it, clipped to
  [0, 2 pi] (the glued point is not crossed), satisfies A x(theta) <= b in
  the likelihood definition of Sec. 2.2.
"""
import math

import numpy as np
import pytest

import oracle

TWO_PI = 2.0 * math.pi


def _arcs_instance(x, nu, arcs):
    """Rows whose infeasible open arc on the ellipse x cos + nu sin is (t1, t2):
    tau = (t1 + t2) / 2, h = (t2 - t1) / 2, (a.x, a.nu) = (cos tau, sin tau),
    b = cos h (the worked-example construction of Sec. 2)."""
    M = np.stack([x, nu])
    A, b = [], []
    for t1, t2 in arcs:
        tau, h = 0.5 * (t1 + t2), 0.5 * (t2 - t1)
        A.append(np.linalg.solve(M, [math.cos(tau), math.sin(tau)]))
        b.append(math.cos(h))
    return np.array(A), np.array(b)


X_T = np.array([1.0, 0.5])
NU = np.array([-2.3, 2.1])
ARCS = [(0.5, 1.0), (1.1, 3.0), (4.0, 5.0)]


@pytest.mark.parametrize("eps,expected", [
    (0.0, [(0.0, 0.5), (1.0, 1.1), (3.0, 4.0), (5.0, TWO_PI)]),
    (0.04, [(0.0, 0.46), (1.04, 1.06), (3.04, 3.96), (5.04, TWO_PI)]),
    # 2 eps > 0.1: the piece [1.0, 1.1] is dropped; 0 and 2 pi stay
    (0.06, [(0.0, 0.44), (3.06, 3.94), (5.06, TWO_PI)]),
    (0.3, [(0.0, 0.2), (3.3, 3.7), (5.3, TWO_PI)]),
])
def test_trim_hand_derived(eps, expected):
    A, b = _arcs_instance(X_T, NU, ARCS)
    r = oracle.step(A, b, X_T, NU, 0.5, trim_eps=eps)
    pieces = r.pieces[r.pieces[:, 1] > r.pieces[:, 0]]
    np.testing.assert_allclose(pieces, np.array(expected), rtol=0, atol=1e-12)
    # theta from the trimmed pieces (inverse CDF over them)
    total = sum(h - l for l, h in expected)
    s = 0.5 * total
    for l, h in expected:
        if s <= h - l:
            assert r.theta == pytest.approx(l + s, abs=1e-12)
            break
        s -= h - l


def test_trim_drops_pieces_one_by_one():
    """Growing eps drops the pieces in order of length; the glued ends 0 and
    2 pi never move, and an empty set gives theta = 0 (stay)."""
    A, b = _arcs_instance(X_T, NU, ARCS)
    r = oracle.step(A, b, X_T, NU, 0.9, trim_eps=0.45)
    np.testing.assert_allclose(r.pieces, [[0.0, 0.05], [3.45, 3.55], [5.45, TWO_PI]],
                               rtol=0, atol=1e-12)
    r = oracle.step(A, b, X_T, NU, 0.9, trim_eps=0.52)
    np.testing.assert_allclose(r.pieces, [[5.52, TWO_PI]], rtol=0, atol=1e-12)
    r = oracle.step(A, b, X_T, NU, 0.9, trim_eps=1.5)
    assert r.pieces.shape[0] == 0 and r.theta == 0.0
    np.testing.assert_array_equal(r.x_next, X_T)


def _trimmed_by_grid(A, b, x, nu, eps, n):
    """Trimmed active set on the grid theta_k = 2 pi k / n: theta_k is in it iff
    every grid angle within eps of it (clipped to [0, 2 pi]) is feasible."""
    th = np.linspace(0.0, TWO_PI, n + 1)
    pts = np.outer(np.cos(th), x) + np.outer(np.sin(th), nu)
    feas = np.all(pts @ A.T <= b[None, :], axis=1)
    w = int(math.floor(eps / (TWO_PI / n)))
    bad = np.concatenate([[0], np.cumsum(~feas)])
    k = np.arange(n + 1)
    lo = np.maximum(0, k - w)
    hi = np.minimum(n, k + w)
    inside = (bad[hi + 1] - bad[lo]) == 0
    return th, inside


def _runs(th, inside):
    out = []
    k = 0
    n = inside.size
    while k < n:
        if inside[k]:
            j = k
            while j + 1 < n and inside[j + 1]:
                j += 1
            out.append((th[k], th[j]))
            k = j + 1
        else:
            k += 1
    return np.array(out).reshape(-1, 2)


@pytest.mark.parametrize("seed", range(12))
def test_trim_brute_force_grid(seed):
    rng = np.random.default_rng(500 + seed)
    d = int(rng.integers(2, 5))
    m = int(rng.integers(1, 7))
    x = rng.standard_normal(d) * 0.3
    A = rng.standard_normal((m, d))
    b = A @ x + rng.uniform(0.05, 1.0, size=m)
    nu = rng.standard_normal(d)
    eps = float(rng.uniform(0.01, 0.3))
    n = 1 << 18
    h = TWO_PI / n
    th, inside = _trimmed_by_grid(A, b, x, nu, eps, n)
    grid_pieces = _runs(th, inside)
    r = oracle.step(A, b, x, nu, 0.3, trim_eps=eps)
    pieces = r.pieces[r.pieces[:, 1] > r.pieces[:, 0]]
    # measure within a few grid spacings per endpoint
    gm = float(np.sum(grid_pieces[:, 1] - grid_pieces[:, 0]))
    om = float(np.sum(pieces[:, 1] - pieces[:, 0]))
    assert abs(gm - om) <= (4 * max(len(pieces), 1) + 4) * h, (gm, om)
    # the same pieces, endpoint by endpoint (pieces longer than a few spacings)
    big = pieces[pieces[:, 1] - pieces[:, 0] > 8 * h]
    gbig = grid_pieces[grid_pieces[:, 1] - grid_pieces[:, 0] > 8 * h]
    assert big.shape == gbig.shape, (big, gbig)
    np.testing.assert_allclose(big, gbig, rtol=0, atol=3 * h)
    # theta lies in the trimmed set
    if pieces.shape[0]:
        assert any(lo - 1e-12 <= r.theta <= hi + 1e-12 for lo, hi in pieces)
