"""FP64 form: one-step map of the CUDA path vs the FP64 oracle, identical draws.

Bar (stated for the plain FP64 form): interval endpoints within 1e-10 rad,
theta within 1e-10 rad, x_{t+1} within 1e-9 relative, identical rejection
flags.  The cases cover the paper's worked examples (Fig. 1, Fig. 2), random
polytopes at sizes that span several GEMM and sort tiles with ragged tails,
forced ties (Sec. 3.1, App. C), the sort reduction (Sec. 3.1), rows without
roots, d = 1, and a single chain.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
from conftest import read_golden
from gpu_helpers import dev, host, oracle_steps, positive_pieces, feasible_instance

pytestmark = pytest.mark.gpu

ANG_TOL = 1e-10
X_RTOL = 1e-9


def run_step(A, b, X, NU, U, precision=ess.ESS_PREC_FP64, max_pieces=None, **cfg):
    s = ess.Sampler(A, b, precision=precision, **cfg)
    try:
        if not cfg.get("sort_threads"):
            # the warp-per-chain kernel (the default picks a CTA per chain for
            # fewer chains than SMs, test_few_chains_take_a_cta_per_chain)
            ess.ess_set_chain_kernel(s.state, ess.ESS_CHAIN_WARP)
        mp = max_pieces or (A.shape[0] + 2)
        Xn, th, pcs, npc, rej = s.step_with_draws(dev(X), dev(NU), dev(U), max_pieces=mp)
        return host(Xn), host(th), host(pcs), host(npc), host(rej), s.stats()
    finally:
        s.close()


def check_fp64(A, b, X, NU, U, trim_eps=0.0, **cfg):
    Xn, th, pcs, npc, rej, _ = run_step(A, b, X, NU, U, trim_eps=trim_eps, **cfg)
    ref = oracle_steps(A, b, X, NU, U, trim_eps)
    for c, r in enumerate(ref):
        assert r.status == 0
        want = positive_pieces(r.pieces)
        got = positive_pieces(pcs[c], min(npc[c], pcs.shape[1]))
        assert npc[c] == want.shape[0], (c, npc[c], want)
        np.testing.assert_allclose(got, want, rtol=0, atol=ANG_TOL)
        assert abs(th[c] - r.theta) <= ANG_TOL, (c, th[c], r.theta)
        assert bool(rej[c]) == r.rejected
        scale = np.maximum(1.0, np.abs(r.x_next))
        assert np.all(np.abs(Xn[c] - r.x_next) <= X_RTOL * scale), c
    return Xn, th


def test_fig1_worked_example():
    rows = read_golden("fig1_worked_example.txt")
    x = np.array([float(v) for v in rows[0][1:]])
    nu = np.array([float(v) for v in rows[1][1:]])
    A, b = [], []
    for row in rows[2:]:
        if row[0] == "plane":
            t1, t2 = float(row[1]) * math.pi, float(row[2]) * math.pi
            tau, h = 0.5 * (t1 + t2), 0.5 * (t2 - t1)
            A.append(np.linalg.solve(np.stack([x, nu]), [math.cos(tau), math.sin(tau)]))
            b.append(math.cos(h))
    A, b = np.array(A), np.array(b)
    U = np.array([0.0, 0.1, 0.35, 0.5, 0.77, 0.999])
    X = np.tile(x, (U.size, 1))
    NU = np.tile(nu, (U.size, 1))
    Xn, th = check_fp64(A, b, X, NU, U)
    _, _, pcs, npc, _, _ = run_step(A, b, X, NU, U)
    expected = np.array([[0.0, 0.125], [0.875, 1.125], [1.75, 2.0]]) * math.pi
    np.testing.assert_allclose(positive_pieces(pcs[0], npc[0]), expected, atol=1e-12)


def test_fig2_edge_cases():
    x = np.array([[2.0, 0.0]])
    nu = np.array([[0.0, 1.0]])
    a = np.array([[-1.0, 0.0]])
    for b_val in (2.5, 2.0, 1.0, -2.0):
        Xn, th, pcs, npc, rej, _ = run_step(a, np.array([b_val]), x, nu, np.array([0.4]))
        r = oracle.step(a, np.array([b_val]), x[0], nu[0], 0.4)
        if b_val == -2.0:
            assert th[0] == 0.0 and npc[0] == 0  # I_act = {0}: stay
            np.testing.assert_array_equal(Xn[0], x[0])
        check_fp64(a, np.array([b_val]), x, nu, np.array([0.4]))
        assert abs(th[0] - r.theta) <= ANG_TOL
    # b/r = -1.25: x_t infeasible -> the API refuses the step
    with pytest.raises(ess.EssError) as e:
        run_step(a, np.array([-2.5]), x, nu, np.array([0.4]))
    assert e.value.status == ess.ESS_ERR_INFEASIBLE_X0


@pytest.mark.parametrize("d,m,n", [(1, 2, 7), (3, 5, 33), (10, 20, 16), (37, 75, 130),
                                   (137, 300, 200), (64, 513, 65), (200, 1100, 40),
                                   (129, 2051, 24)])
def test_random_polytopes(d, m, n):
    rng = np.random.default_rng(1000 * d + m)
    A, b, X = feasible_instance(rng, d, m, n)
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    check_fp64(A, b, X, NU, U)


def test_ties_and_duplicate_rows():
    rng = np.random.default_rng(8)
    d, m, n = 6, 40, 50
    A, b, X = feasible_instance(rng, d, m, n)
    A[10:20] = A[0]          # identical rows: identical (alpha, beta)
    b[10:20] = b[0]
    A[20:25] = A[1] * 2.0    # parallel rows, same hyperplane: identical angles
    b[20:25] = b[1] * 2.0
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    check_fp64(A, b, X, NU, U)


def test_rows_without_roots_and_whole_circle():
    rng = np.random.default_rng(9)
    d, m, n = 5, 30, 20
    A = rng.standard_normal((m, d))
    b = np.full(m, 1e6)      # every b/r > 1: I_act = [0, 2 pi]
    X = np.zeros((n, d))
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    Xn, th = check_fp64(A, b, X, NU, U)
    np.testing.assert_allclose(th, 2 * math.pi * U, atol=1e-12)


def test_sort_reduction_through_kernel():
    """Sec. 3.1: pairs (c_i, c_i + eps) come back in sorted order."""
    # d = 2, x = (1, 0), nu = (0, 1): the ellipse is the unit circle at angle
    # theta; the halfspace cos(theta - tau_i) <= cos(h_i) has infeasible arc
    # (tau_i - h_i, tau_i + h_i).
    rng = np.random.default_rng(12)
    c = np.sort(rng.uniform(0.2, 2 * math.pi - 0.3, size=600))
    rng.shuffle(c)
    eps = 0.25 * np.min(np.diff(np.sort(c)))
    tau, h = c + eps / 2, np.full_like(c, eps / 2)
    A = np.stack([np.cos(tau), np.sin(tau)], axis=1)
    b = np.cos(h)
    x = np.array([[1.0, 0.0]])
    nu = np.array([[0.0, 1.0]])
    _, _, pcs, npc, _, _ = run_step(A, b, x, nu, np.array([0.5]), max_pieces=700)
    got = positive_pieces(pcs[0], npc[0])
    order = np.sort(c)
    assert got.shape[0] == c.size + 1
    np.testing.assert_allclose(got[1:-1, 1], order[1:], atol=1e-12)
    np.testing.assert_allclose(got[1:-1, 0], order[:-1] + eps, atol=1e-12)


def test_rows_beyond_float_range():
    """FP64 chains classify rows in FP32 (integer double-to-float rounding):
    rows scaled by 1e40 (p, q, b overflow float) and by 1e-41 (they vanish
    in float) are kept for exact FP64 roots, so the step still equals the
    oracle's; the halfspaces are the unscaled ones, so the pieces are too."""
    rng = np.random.default_rng(41)
    d, m, n = 7, 60, 40
    A, b, X = feasible_instance(rng, d, m, n)
    A[:12] *= 1e40
    b[:12] *= 1e40
    A[12:24] *= 1e-41
    b[12:24] *= 1e-41
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    for sort_threads in (0, 256):
        check_fp64(A, b, X, NU, U, sort_threads=sort_threads)


def test_single_chain_and_trim():
    rng = np.random.default_rng(13)
    A, b, X = feasible_instance(rng, 12, 40, 1)
    NU = rng.standard_normal((1, 12))
    for u in (0.0, 0.3, 0.9999):
        check_fp64(A, b, X, NU, np.array([u]))
    X2 = np.repeat(X, 30, axis=0)
    NU2 = rng.standard_normal((30, 12))
    check_fp64(A, b, X2, NU2, rng.uniform(size=30), trim_eps=1e-3)


def test_full_size_sampled_chains():
    """The d = 1000, m = 2000, 8192-chain workload in the benchmark's launch,
    checked on 24 sampled chains against the oracle."""
    import workloads
    inst = workloads.metric(n_chains=8192)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((8192, inst.d)) * 0.002  # feasible: |a.x| small vs b >= 0.05
    assert np.max(X @ inst.A.T - inst.b) < 0
    NU = rng.standard_normal((8192, inst.d))
    U = rng.uniform(size=8192)
    Xn, th, pcs, npc, rej, _ = run_step(inst.A, inst.b, X, NU, U, max_pieces=64)
    idx = rng.choice(8192, size=24, replace=False)
    ref = oracle_steps(inst.A, inst.b, X[idx], NU[idx], U[idx])
    for k, c in enumerate(idx):
        r = ref[k]
        assert abs(th[c] - r.theta) <= ANG_TOL
        np.testing.assert_allclose(positive_pieces(pcs[c], min(npc[c], 64)),
                                   positive_pieces(r.pieces)[:64], atol=ANG_TOL)
        assert np.all(np.abs(Xn[c] - r.x_next) <= X_RTOL * np.maximum(1, np.abs(r.x_next)))
    # every chain: the emitted iterate is feasible in FP64
    assert np.max(Xn @ inst.A.T - inst.b) <= 0.0


@pytest.mark.parametrize("sort_threads", [0, 256])
def test_both_step_kernels(sort_threads):
    """The warp-per-chain kernel (default) and the CTA-per-chain kernel give the
    oracle's step on the same inputs, including a probit-style orthant (equal
    half-widths, b = 0) where no arc contains another: the warp kernel keeps
    only the extremes of the long arcs' union, the CTA kernel merges them all."""
    rng = np.random.default_rng(21)
    d, m, n = 40, 600, 96
    A, b, X = feasible_instance(rng, d, m, n)
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    check_fp64(A, b, X, NU, U, sort_threads=sort_threads)
    # a probit-style orthant (A = -diag(y) L, b = 0): every arc has half-width
    # pi / 2 and no arc contains another; together they form one arc
    M = rng.standard_normal((200, 200))
    L = np.linalg.cholesky(M @ M.T / 200 + np.eye(200))
    z = rng.standard_normal(200)
    y = np.sign(L @ z)
    A2 = -y[:, None] * L
    b2 = np.zeros(200)
    X2 = np.tile(z, (32, 1))
    check_fp64(A2, b2, X2, rng.standard_normal((32, 200)), rng.uniform(size=32),
               sort_threads=sort_threads)


@pytest.mark.parametrize("sort_threads", [0, 256])
def test_cta_kernel_short_arcs(sort_threads):
    """Arcs shorter than a bucket of the CTA kernel's interval merge (half-width
    1e-3 rad against buckets of 2 pi / 512 in FP64) make it sort the arcs instead; the
    step still equals the oracle's.  The other chains' arcs are merged per
    bucket (long arcs only)."""
    rng = np.random.default_rng(33)
    d, m_long, m_short, n = 12, 300, 24, 8
    x = rng.standard_normal(d) * 0.2
    nu = rng.standard_normal(d)
    A_long = rng.standard_normal((m_long, d))
    b_long = A_long @ x + rng.uniform(0.2, 1.0, size=m_long)
    A_short, b_short = [], []
    while len(A_short) < m_short:
        a = rng.standard_normal(d)
        p, q = a @ x, a @ nu
        r = math.hypot(p, q)
        bb = r * math.cos(1e-3)
        if p < bb - 1e-9 * r:  # x strictly feasible: the short arc avoids 0
            A_short.append(a)
            b_short.append(bb)
    A = np.vstack([A_long, np.array(A_short)])
    b = np.concatenate([b_long, np.array(b_short)])
    X = np.tile(x, (n, 1))
    NU = np.tile(nu, (n, 1))
    U = np.linspace(0.05, 0.95, n)
    check_fp64(A, b, X, NU, U, sort_threads=sort_threads)
    # the long-arc rows alone take the bucket merge in the CTA kernel
    check_fp64(A_long, b_long, X, NU, U, sort_threads=sort_threads)


@pytest.mark.parametrize("precision", [ess.ESS_PREC_FP64, ess.ESS_PREC_MIXED])
def test_few_chains_take_a_cta_per_chain(precision):
    """ESS_CHAIN_AUTO with fewer chains than SMs (m > 256) steps each chain
    with a CTA (its rows over the CTA's threads) instead of one warp: the
    kernel reported for the loaded chains, and the step against the oracle."""
    import torch
    rng = np.random.default_rng(41)
    d, m, n = 30, 700, 10
    A, b, X = feasible_instance(rng, d, m, n, scale=1.0 / math.sqrt(d), slack=(0.1, 1.0))
    s = ess.Sampler(A, b, precision=precision)
    try:
        ess.ess_chains_init(s.state, dev(X), n, 0)
        assert ess.ess_get_chain_kernel(s.state) == ess.ESS_CHAIN_CTA
        ess.ess_set_chain_kernel(s.state, ess.ESS_CHAIN_WARP)
        assert ess.ess_get_chain_kernel(s.state) == ess.ESS_CHAIN_WARP
    finally:
        s.close()
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    if precision == ess.ESS_PREC_FP64:
        Xn, th, pcs, npc, rej, _ = run_step(A, b, X, NU, U, sort_threads=0)  # warp
        s = ess.Sampler(A, b, precision=precision)
        try:
            got = s.step_with_draws(dev(X), dev(NU), dev(U), max_pieces=m + 2)
            Xa, tha = host(got[0]), host(got[1])
        finally:
            s.close()
        ref = oracle_steps(A, b, X, NU, U, 0.0)
        for c, r in enumerate(ref):
            assert abs(tha[c] - r.theta) <= ANG_TOL, (c, tha[c], r.theta)
            assert np.all(np.abs(Xa[c] - r.x_next) <= X_RTOL * np.maximum(1.0, np.abs(r.x_next)))

