"""Chains with m beyond the CTA kernel's 8192 arcs (Sec. 3.1 sorts all 2m
angles of a chain; here m reaches 20000): the warp kernel takes the chains
whose arcs mostly drop out in the domination prune, and the wide-row kernel
(rows streamed, arcs merged per bucket, short arcs and the sort spilled to
global scratch when they outgrow shared memory) takes the rest -- or every
chain with sort_threads > 0.  Each case is compared with the FP64 oracle's
one-step map, element by element: the FP64 form to 1e-10 rad (pieces, theta)
and 1e-9 relative (x'), the mixed form on grid inputs (exact products) to
1e-5 rad with the a-priori exemptions of gpu_helpers.

Instances:
  * a random polytope (most chains pruned to a few arcs: the warp kernel);
  * cones through x's side of the origin (b = 0): every arc has half-width
    pi / 2 and no arc contains another, so all arcs survive the prune and
    every chain overflows to the wide-row kernel, whose bucket merge keeps
    them in shared memory;
  * a circle of near-tangent rows (d = 2, x = e1, nu = e2: the ellipse is the
    unit circle and row i cuts the arc (phi_i - h, phi_i + h) with h = 2e-4,
    shorter than a merge bucket): thousands of short arcs, more than shared
    memory holds, so the arcs go through the global merge sort and the
    chunked Alg. 3.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
from gpu_helpers import dev, host, oracle_steps, positive_pieces, feasible_instance, f32, \
    grid_bits, to_grid, mixed_endpoint_bounds, mixed_exempt, merge

pytestmark = pytest.mark.gpu

ANG64, XR64 = 1e-10, 1e-9
ANG32 = 1e-5


def _sym_diff(p1, p2):
    """|P1 symmetric-difference P2| for unions of closed intervals, by one
    sweep over the two merged (sorted, disjoint) lists."""
    a, b = merge(p1), merge(p2)
    inter, i, j = 0.0, 0, 0
    while i < len(a) and j < len(b):
        lo, hi = max(a[i, 0], b[j, 0]), min(a[i, 1], b[j, 1])
        inter += max(0.0, hi - lo)
        if a[i, 1] < b[j, 1]:
            i += 1
        else:
            j += 1
    meas = lambda p: float(np.sum(p[:, 1] - p[:, 0])) if len(p) else 0.0
    return meas(a) + meas(b) - 2.0 * inter


def _run(A, b, X, NU, U, precision, max_pieces, warp_first=False, **cfg):
    s = ess.Sampler(A, b, precision=precision, **cfg)
    try:
        if warp_first:
            ess.ess_set_chain_kernel(s.state, ess.ESS_CHAIN_WARP)
            assert ess.ess_get_chain_kernel(s.state) == (
                ess.ESS_CHAIN_CTA if cfg.get("sort_threads") else ess.ESS_CHAIN_WARP)
        else:
            if np.any(b <= 0.0):
                # rows with b <= 0 make the default run the warp kernel first;
                # ESS_CHAIN_STREAM keeps the wide-row kernel for every chain
                ess.ess_set_chain_kernel(s.state, ess.ESS_CHAIN_STREAM)
            assert ess.ess_get_chain_kernel(s.state) == ess.ESS_CHAIN_CTA
        Xn, th, pcs, npc, rej = s.step_with_draws(dev(X), dev(NU), dev(U), max_pieces=max_pieces)
        out = host(Xn), host(th), host(pcs), host(npc), host(rej), s.stats()
        m_max, _ = ess.ess_limits(s.state)
    finally:
        s.close()
    assert m_max >= A.shape[0]
    return out


def check_fp64(A, b, X, NU, U, max_pieces, warp_first=False, **cfg):
    Xn, th, pcs, npc, rej, st = _run(A, b, X, NU, U, ess.ESS_PREC_FP64, max_pieces, warp_first,
                                     **cfg)
    refs = oracle_steps(A, b, X, NU, U)
    for c, r in enumerate(refs):
        want = positive_pieces(r.pieces)
        assert npc[c] == want.shape[0], (c, npc[c], want.shape[0])
        got = positive_pieces(pcs[c], min(npc[c], pcs.shape[1]))
        if want.shape[0] <= pcs.shape[1]:
            np.testing.assert_allclose(got, want, rtol=0, atol=ANG64)
        assert abs(th[c] - r.theta) <= ANG64, (c, th[c], r.theta)
        assert bool(rej[c]) == r.rejected
        assert np.all(np.abs(Xn[c] - r.x_next) <= XR64 * np.maximum(1.0, np.abs(r.x_next))), c
    assert np.max(Xn @ A.T - b) <= 0.0
    return st


def check_mixed(A, b, X, NU, U, max_pieces, max_exempt_frac=0.05, warp_first=False, **cfg):
    X, NU = f32(X), f32(NU)
    refs = oracle_steps(A, b, X, NU, U)
    amp, arith = mixed_endpoint_bounds(A, b, X, NU)
    exempt = mixed_exempt(refs, amp, arith, 0.5 * ANG32)
    Xn, th, pcs, npc, rej, st = _run(A, b, X, NU, U, ess.ESS_PREC_MIXED, max_pieces, warp_first,
                                     **cfg)
    assert np.max(Xn @ A.T - b) <= 0.0
    for c, r in enumerate(refs):
        if exempt[c]:
            continue
        want = positive_pieces(r.pieces)
        got = positive_pieces(pcs[c], min(npc[c], pcs.shape[1]))
        if want.shape[0] <= pcs.shape[1]:
            assert _sym_diff(got, want) <= 2 * max(len(want), 1) * ANG32, c
            if got.shape == want.shape:
                assert np.max(np.abs(got - want), initial=0.0) <= ANG32, c
        assert abs(th[c] - r.theta) <= ANG32, (c, th[c], r.theta)
        if rej[c]:
            np.testing.assert_array_equal(Xn[c], X[c])
        else:
            assert np.all(np.abs(Xn[c] - r.x_next)
                          <= ANG32 * (1 + np.abs(r.x_next)) * (1 + np.abs(NU[c]))), c
    assert exempt.sum() <= max_exempt_frac * len(refs)
    return st


def _cones(rng, d, m, n, grid=False):
    """Rows a_i with a_i . x0 < 0, b = 0: every arc has half-width pi / 2."""
    x0 = rng.standard_normal(d)
    A = rng.standard_normal((m, d))
    if grid:
        A = to_grid(A, grid_bits(d))
        x0 = to_grid(x0, grid_bits(d))
    A = -np.sign(A @ x0)[:, None] * A
    keep = (A @ x0) < 0
    A = A[keep]
    X = np.tile(x0, (n, 1))
    NU = rng.standard_normal((n, d))
    if grid:
        NU = to_grid(NU, grid_bits(d))
    return A, np.zeros(A.shape[0]), X, NU


def _circle(rng, m, h=2e-4, grid=False):
    """d = 2, x = e1, nu = e2; row i is the direction phi_i scaled so that
    b_i / r_i = cos(h): the infeasible arc (phi_i - h, phi_i + h)."""
    phi = np.sort(rng.uniform(0.01, 2 * math.pi - 0.01, size=m))
    A = np.stack([np.cos(phi), np.sin(phi)], axis=1)
    if grid:
        A = np.unique(np.round(A * 2040.0), axis=0) / 2048.0
        rng.shuffle(A)
    r = np.hypot(A[:, 0], A[:, 1])
    b = r * math.cos(h)
    keep = A[:, 0] < b - 1e-9 * r   # x = e1 strictly feasible
    return A[keep], b[keep]


# (sort_threads, warp_first): the wide-row kernel for every chain (the
# default), the warp kernel first with the wide-row kernel for the chains it
# leaves, and sort_threads > 0
PATHS = [(0, False), (0, True), (256, False)]


@pytest.mark.parametrize("sort_threads,warp_first", PATHS)
def test_wide_fp64_random_polytope(sort_threads, warp_first):
    rng = np.random.default_rng(1)
    d, m, n = 24, 17001, 40
    A, b, X = feasible_instance(rng, d, m, n, scale=1.0 / math.sqrt(d), slack=(0.05, 0.6))
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    check_fp64(A, b, X, NU, U, max_pieces=256, sort_threads=sort_threads, warp_first=warp_first)


@pytest.mark.parametrize("sort_threads,warp_first", PATHS)
def test_wide_fp64_cones_every_arc_survives(sort_threads, warp_first):
    rng = np.random.default_rng(2)
    A, b, X, NU = _cones(rng, 16, 12000, 12)
    U = rng.uniform(size=X.shape[0])
    st = check_fp64(A, b, X, NU, U, max_pieces=64, sort_threads=sort_threads,
                    warp_first=warp_first)
    # every arc reached the interval merge (no arc contains another)
    assert st["sort_keys"] >= X.shape[0]


def test_wide_fp64_short_arcs_global_sort():
    rng = np.random.default_rng(3)
    A, b = _circle(rng, 12000)
    n = 6
    X = np.tile([1.0, 0.0], (n, 1))
    NU = np.tile([0.0, 1.0], (n, 1))
    U = np.array([0.0, 0.13, 0.5, 0.71, 0.9, 0.999])
    st = check_fp64(A, b, X, NU, U, max_pieces=A.shape[0] + 2)
    # all but a few arcs are shorter than a bucket: more than shared memory holds
    assert st["sort_keys"] > 6 * 8000


def test_wide_fp64_short_and_long_arcs_smem():
    """A few hundred short arcs (half-width 1e-4) among cones: the short list
    stays in shared memory and is sorted with the bucket intervals."""
    rng = np.random.default_rng(4)
    d = 10
    A0, b0, X, NU = _cones(rng, d, 9500, 8)
    x, nu = X[0], NU[0]
    extra, bs = [], []
    while len(extra) < 300:
        a = rng.standard_normal(d)
        p, q = a @ x, a @ nu
        r = math.hypot(p, q)
        bb = r * math.cos(1e-4)
        if p < bb - 1e-9 * r:
            extra.append(a)
            bs.append(bb)
    A = np.vstack([A0, np.array(extra)])
    b = np.concatenate([b0, np.array(bs)])
    NUt = np.tile(nu, (8, 1))
    U = np.linspace(0.02, 0.98, 8)
    check_fp64(A, b, X, NUt, U, max_pieces=512)


@pytest.mark.parametrize("sort_threads,warp_first", PATHS)
def test_wide_mixed_cones(sort_threads, warp_first):
    rng = np.random.default_rng(5)
    A, b, X, NU = _cones(rng, 16, 10000, 16, grid=True)
    U = rng.uniform(size=X.shape[0])
    check_mixed(A, b, X, NU, U, max_pieces=64, sort_threads=sort_threads, warp_first=warp_first)


@pytest.mark.parametrize("warp_first", [False, True])
def test_wide_mixed_random_grid(warp_first):
    rng = np.random.default_rng(6)
    d, m, n = 32, 20011, 64
    B = grid_bits(d)
    A = to_grid(rng.standard_normal((m, d)) / math.sqrt(d), B)
    X = to_grid(rng.standard_normal((n, d)) * 0.3, B)
    NU = to_grid(rng.standard_normal((n, d)), B)
    b = (X @ A.T).max(axis=0) + rng.uniform(0.05, 0.6, size=m)
    U = rng.uniform(size=n)
    check_mixed(A, b, X, NU, U, max_pieces=256, warp_first=warp_first)


def test_wide_mixed_short_arcs_global_sort():
    """Grid directions (exact p and q in the mixed form); b / r = cos(2e-4)
    puts every row in the FP64 near-tangent branch, so the endpoints match the
    oracle to FP64 rounding."""
    rng = np.random.default_rng(7)
    A, b = _circle(rng, 20000, grid=True)
    assert A.shape[0] > 8000
    n = 4
    X = np.tile([1.0, 0.0], (n, 1))
    NU = np.tile([0.0, 1.0], (n, 1))
    U = np.array([0.05, 0.4, 0.6, 0.95])
    st = check_mixed(A, b, X, NU, U, max_pieces=A.shape[0] + 2, max_exempt_frac=0.0)
    assert st["tangent_fp64"] >= n * A.shape[0]


def test_wide_run_feasible_and_matches_oracle_run():
    """ess_run (drawn nu and theta, p carried between refreshes) at m = 10000:
    8 steps against the oracle's 8 steps with the same Philox counters."""
    rng = np.random.default_rng(8)
    d, m, n = 20, 10000, 16
    A, b, X0 = feasible_instance(rng, d, m, n, scale=1.0 / math.sqrt(d), slack=(0.05, 0.6))
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_FP64)
    try:
        X = dev(X0)
        s.run(X, 8, seed=5)
        Xg = host(X)
    finally:
        s.close()
    want = oracle.run(A, b, X0, 8, seed=5)[0]
    gap = np.max(np.abs(Xg - want) / np.maximum(1.0, np.abs(want)), axis=1)
    assert np.all(gap <= 1e-9), gap
    assert np.max(Xg @ A.T - b) <= 0.0


def test_wide_limits_and_beyond():
    s = ess.Sampler(np.eye(2), np.ones(2), precision=ess.ESS_PREC_MIXED)
    try:
        m_max, d_max = ess.ess_limits(s.state)
    finally:
        s.close()
    assert m_max == 1 << 22
    rng = np.random.default_rng(9)
    A = rng.standard_normal((9000, 8))
    s = ess.Sampler(A, np.ones(9000) * 10.0, precision=ess.ESS_PREC_FP64)
    try:
        m_w, d_w = ess.ess_limits(s.state)
        assert m_w == 1 << 22 and d_w > 1000
    finally:
        s.close()
