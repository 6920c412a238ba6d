"""Pins of the oracle's roots and active-interval construction.

Each test checks the FP64 oracle against something the paper or plain
mathematics fixes, never against the oracle itself:

* Fig. 2 edge-case gallery (Sec. 3.2) -- printed geometry, exact angles.
* Eq. trigonometry-equation by substitution (App. B) -- the returned angles
  must solve p cos(theta) + q sin(theta) = b, with the infeasible side inside.
* Fig. 1 worked example (Sec. 2) -- active intervals printed in the caption.
* App. D worst case -- closed-form k+1 pieces.
* Sec. 3.1 sort reduction -- the pieces reveal the sorted order.
* A dense theta-grid brute force of the likelihood definition (Sec. 2.2) on
  tiny random instances, including forced ties (Sec. 3.1, App. C).
"""
import math

import numpy as np
import pytest

import oracle
from conftest import read_golden

PI = math.pi


def _merge(pieces, tol=0.0):
    """Union of closed pieces as disjoint positive-length intervals."""
    out = []
    for lo, hi in sorted((float(a), float(b)) for a, b in pieces):
        if hi - lo <= tol:
            continue
        if out and lo <= out[-1][1] + tol:
            out[-1][1] = max(out[-1][1], hi)
        else:
            out.append([lo, hi])
    return out


# --------------------------------------------------------------------------
# Fig. 2 gallery
# --------------------------------------------------------------------------

def test_fig2_edge_cases():
    rows = read_golden("fig2_edge_cases.txt")
    x = np.array([float(v) for v in rows[0][1:]])
    nu = np.array([float(v) for v in rows[1][1:]])
    a = np.array([float(v) for v in rows[2][1:]])
    p, q = float(a @ x), float(a @ nu)
    assert (p, q) == (-2.0, 0.0)
    for row in rows[3:]:
        b, ratio, kind = float(row[1]), float(row[2]), row[3]
        assert b / math.hypot(p, q) == pytest.approx(ratio)
        k, alpha, beta = oracle.roots(p, q, b)
        if kind == "none":
            assert k == 0
        elif kind == "arc":
            assert k == 1
            assert alpha == pytest.approx(float(row[4]) * PI, abs=1e-14)
            assert beta == pytest.approx(float(row[5]) * PI, abs=1e-14)
        else:
            # x_t violates a.x <= b: the one-step map must report it
            res = oracle.step(a.reshape(1, 2), np.array([b]), x, nu, 0.5)
            assert res.status == -1


def test_fig2_b_minus_r_gives_single_point():
    # b/r = -1 (Fig. 2d): I_act is the glued point {0, 2 pi}; theta must be 0.
    a = np.array([[-1.0, 0.0]])
    res = oracle.step(a, np.array([-2.0]), np.array([2.0, 0.0]), np.array([0.0, 1.0]), 0.73)
    assert res.theta == 0.0
    assert np.array_equal(res.x_next, [2.0, 0.0])
    assert not res.rejected
    assert sum(hi - lo for lo, hi in res.pieces) == 0.0


# --------------------------------------------------------------------------
# App. B: substitution into the trigonometric equation
# --------------------------------------------------------------------------

def test_roots_solve_equation_and_orient_arc():
    rng = np.random.default_rng(1)
    n_checked = 0
    for _ in range(20000):
        p, q = rng.standard_normal(2) * rng.choice([1e-3, 1.0, 1e3])
        r = math.hypot(p, q)
        b = p + abs(rng.standard_normal()) * r  # feasible: p <= b
        k, alpha, beta = oracle.roots(p, q, b)
        if b / r >= 1.0:
            assert k == 0
            continue
        assert k == 1
        assert 0.0 <= alpha < beta <= 2 * PI
        scale = r
        for th in (alpha, beta):
            assert abs(p * math.cos(th) + q * math.sin(th) - b) <= 1e-12 * scale + 1e-12 * abs(b)
        mid = 0.5 * (alpha + beta)
        assert p * math.cos(mid) + q * math.sin(mid) > b      # inside: violated
        # outside the arc, near each end: satisfied
        h = 1e-6 * (beta - alpha)
        if alpha - h > 0:
            assert p * math.cos(alpha - h) + q * math.sin(alpha - h) <= b + 1e-12 * scale
        if beta + h < 2 * PI:
            assert p * math.cos(beta + h) + q * math.sin(beta + h) <= b + 1e-12 * scale
        n_checked += 1
    assert n_checked > 5000


def test_roots_no_root_cases():
    assert oracle.roots(0.0, 0.0, 0.3)[0] == 0          # r = 0, tautology
    assert oracle.roots(0.0, 0.0, -0.3)[0] == -1        # r = 0, invalid
    assert oracle.roots(0.3, 0.4, 0.5)[0] == 0          # b / r = 1
    assert oracle.roots(0.3, 0.4, 0.7)[0] == 0          # b / r > 1


# --------------------------------------------------------------------------
# Fig. 1 worked example
# --------------------------------------------------------------------------

def _plane_from_angles(x, nu, t1, t2):
    """Halfspace a.y <= b whose boundary meets the ellipse at t1 < t2, with the
    open arc (t1, t2) on the infeasible side: unit r, tau = (t1 + t2) / 2,
    h = (t2 - t1) / 2, so (p, q) = (cos tau, sin tau) and b = cos h; a solves
    [x nu]^T a = (p, q)."""
    tau, h = 0.5 * (t1 + t2), 0.5 * (t2 - t1)
    M = np.stack([x, nu])
    a = np.linalg.solve(M, np.array([math.cos(tau), math.sin(tau)]))
    return a, math.cos(h)


def _fig1():
    rows = read_golden("fig1_worked_example.txt")
    x = np.array([float(v) for v in rows[0][1:]])
    nu = np.array([float(v) for v in rows[1][1:]])
    A, b, expected = [], [], []
    length = None
    for row in rows[2:]:
        if row[0] == "plane":
            a, bb = _plane_from_angles(x, nu, float(row[1]) * PI, float(row[2]) * PI)
            A.append(a)
            b.append(bb)
        elif row[0] == "piece":
            expected.append((float(row[1]) * PI, float(row[2]) * PI))
        elif row[0] == "length":
            length = float(row[1]) * PI
    return x, nu, np.array(A), np.array(b), expected, length


def test_fig1_worked_example_pieces():
    x, nu, A, b, expected, length = _fig1()
    # x_t itself is feasible
    assert np.all(A @ x <= b)
    res = oracle.step(A, b, x, nu, 0.5)
    assert res.status == 0
    got = _merge(res.pieces)
    assert len(got) == len(expected)
    for (glo, ghi), (elo, ehi) in zip(got, expected):
        assert glo == pytest.approx(elo, abs=1e-12)
        assert ghi == pytest.approx(ehi, abs=1e-12)
    total = sum(hi - lo for lo, hi in res.pieces)
    assert total == pytest.approx(length, abs=1e-12)
    # the third hyperplane's roots are inactive: they are no piece endpoint
    ends = {round(v, 9) for pc in got for v in pc}
    assert round(0.4 * PI, 9) not in ends and round(0.8 * PI, 9) not in ends


def test_fig1_brute_force_grid_agrees():
    x, nu, A, b, expected, length = _fig1()
    theta = np.linspace(0.0, 2 * PI, 2_000_001)
    pts = np.outer(np.cos(theta), x) + np.outer(np.sin(theta), nu)
    feas = np.all(pts @ A.T <= b, axis=1)
    measure = feas.mean() * 2 * PI
    assert measure == pytest.approx(length, abs=1e-4)


# --------------------------------------------------------------------------
# App. D: worst case for Alg. 2, closed form with k + 1 pieces
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 5, 12, 25])
def test_appD_worst_case_closed_form(k):
    i = np.arange(1, k + 1, dtype=np.float64)
    alpha = 2 * PI * (1.0 / 3.0) ** i
    beta = 2 * PI * 2.0 * (1.0 / 3.0) ** i
    got = oracle.active_intervals(alpha, beta)
    expected = [(0.0, 2 * PI * (1 / 3) ** k)]
    expected += [(2 * PI * 2 * (1 / 3) ** j, 2 * PI * (1 / 3) ** (j - 1)) for j in range(k, 0, -1)]
    assert got.shape[0] == k + 1
    for (glo, ghi), (elo, ehi) in zip(got, expected):
        assert glo == pytest.approx(elo, rel=1e-13, abs=1e-300)
        assert ghi == pytest.approx(ehi, rel=1e-13)


# --------------------------------------------------------------------------
# Sec. 3.1 reduction: sorting -> active intervals
# --------------------------------------------------------------------------

def test_sort_reduction_reveals_order():
    rng = np.random.default_rng(7)
    c = rng.uniform(0.1, 2 * PI - 0.1, size=200)
    eps = 0.25 * np.min(np.diff(np.sort(c)))
    got = oracle.active_intervals(c, c + eps)
    order = np.sort(c)
    assert got.shape[0] == c.size + 1
    assert got[0, 0] == 0.0 and got[0, 1] == order[0]
    for kk in range(1, c.size):
        assert got[kk, 0] == order[kk - 1] + eps  # predecessor revealed
        assert got[kk, 1] == order[kk]
    assert got[-1, 0] == order[-1] + eps and got[-1, 1] == 2 * PI


# --------------------------------------------------------------------------
# Likelihood-definition brute force on tiny random instances (with ties)
# --------------------------------------------------------------------------

def _random_feasible_instance(rng, d, m):
    A = rng.standard_normal((m, d))
    x = rng.standard_normal(d) * 0.5
    b = A @ x + rng.uniform(0.0, 1.0, size=m)
    nu = rng.standard_normal(d) * 1.5
    return A, b, x, nu


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_grid_tiny(seed):
    rng = np.random.default_rng(100 + seed)
    d = int(rng.integers(1, 5))
    m = int(rng.integers(1, 9))
    A, b, x, nu = _random_feasible_instance(rng, d, m)
    if seed % 3 == 0 and m >= 2:
        # force a tie: duplicate a row (identical alpha and beta)
        A[1] = A[0]
        b[1] = b[0]
    res = oracle.step(A, b, x, nu, 0.3)
    assert res.status == 0
    n = 1_000_000
    theta = (np.arange(n) + 0.5) * (2 * PI / n)
    P = np.cos(theta)[:, None] * (A @ x)[None, :] + np.sin(theta)[:, None] * (A @ nu)[None, :]
    feas = np.all(P <= b[None, :], axis=1)
    measure = feas.sum() * (2 * PI / n)
    total = sum(hi - lo for lo, hi in res.pieces)
    assert total == pytest.approx(measure, abs=4 * 2 * PI / n * (m + 1))
    # grid points well inside a piece are feasible, well outside are not
    inside = np.zeros(n, dtype=bool)
    for lo, hi in res.pieces:
        inside |= (theta >= lo) & (theta <= hi)
    margin = 1e-9
    near = np.zeros(n, dtype=bool)
    for lo, hi in res.pieces:
        near |= (np.abs(theta - lo) < margin) | (np.abs(theta - hi) < margin)
    assert np.array_equal(inside[~near], feas[~near])


def test_theta_zero_always_active_and_tail_head():
    rng = np.random.default_rng(5)
    for _ in range(300):
        d = int(rng.integers(1, 6))
        m = int(rng.integers(1, 30))
        A, b, x, nu = _random_feasible_instance(rng, d, m)
        res = oracle.step(A, b, x, nu, float(rng.uniform()))
        pcs = res.pieces
        assert pcs[0, 0] == 0.0                       # theta = 0 is in I_act
        assert pcs[-1, 1] == 2 * PI                   # ... and so is 2 pi
        has = res.has_root
        if has.any():
            # Prop. 1, part one: the head piece is [0, min alpha]
            assert pcs[0, 1] == pytest.approx(res.alpha[has].min(), abs=0)
            # part three: the tail piece is [max beta, 2 pi]
            assert pcs[-1, 0] == pytest.approx(res.beta[has].max(), abs=0)
        # theta lies in a piece and x_next is feasible
        assert any(lo <= res.theta <= hi for lo, hi in pcs)
        assert oracle.max_residual(A, b, res.x_next) <= 0.0
