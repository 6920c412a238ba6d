"""Batched problems in one persistent launch per refresh period
(ess_batch_set_persistent): the cooperative kernel that runs the grouped q
GEMM on the tensor cores, the draws of the next step, the warp-per-chain steps
from a device work queue (each after a bounded wait for its problem's q
items, counted by the GEMM's epilogue) and the overflow chains (CTA per
chain), steps joined by bounded grid barriers.

It changes how the work of a step is scheduled, not what is computed: the
chains must equal, bit for bit, those of the graph of per-step launches, which
the batch tests hold against the oracle.  The specs mix uneven d, m and chain
counts (a problem with no chains, d = 1, items crossing the 128-row and
64-chain tiles) with a nearly conic problem (b = 1e-3 on rows that face away
from the start points): every arc is a little shorter than a half circle and
no arc contains another, so every chain keeps more arcs than a warp sorts and
takes the overflow phase.
"""
import math

import numpy as np
import pytest

import paper_2407_10449_gb300 as ess
from gpu_helpers import feasible_instance, host, long_arc_instance

pytestmark = pytest.mark.gpu

# (d, m, chains)
SPECS = [(1, 2, 3), (3, 5, 4), (10, 20, 16), (17, 60, 70), (40, 130, 9), (64, 64, 0),
         (33, 100, 65), (120, 400, 33)]


def cone_instance(rng, d, m, n):
    """{x : A x <= 1e-3} with rows turned to face away from a point x0
    inside, and start points on the ray through x0 (positive multiples stay
    inside).  b > 0 keeps every arc shorter than pi (arcs of b <= 0 form one
    union that the warp step reduces to its two extremes)."""
    x0 = rng.standard_normal(d)
    A = rng.standard_normal((m, d)) / math.sqrt(d)
    A[A @ x0 > 0] *= -1.0
    A[np.abs(A @ x0) < 1e-3] = -x0 / np.linalg.norm(x0)  # no row through x0
    X = x0[None, :] * rng.uniform(0.5, 2.0, size=(n, 1))
    return A, np.full(m, 1e-3), X


def make_batch(seed, with_cone=True):
    rng = np.random.default_rng(seed)
    As, bs, Xs, nc = [], [], [], []
    for d, m, n in SPECS:
        A, b, X = feasible_instance(rng, d, m, max(n, 1), scale=1.0 / math.sqrt(d),
                                    slack=(0.1, 1.0))
        As.append(A)
        bs.append(b)
        Xs.append(X[:n])
        nc.append(n)
    if with_cone:
        A, b, X = cone_instance(rng, 24, 300, 12)
        As.append(A)
        bs.append(b)
        Xs.append(X)
        nc.append(12)
    return As, bs, Xs, nc


def run_batch(As, bs, Xs, nc, persistent, n_iter, t0, refresh_k=4, seed=11):
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED, refresh_k=refresh_k)
    try:
        ess.ess_batch_set_persistent(bs_.batch, persistent)
        X = bs_.pack(Xs)
        bs_.run(nc, X, n_iter, seed=seed, t0=t0)
        return host(X), bs_.stats(), ess.ess_batch_info(bs_.batch)
    finally:
        bs_.close()


def test_persistent_periods_equal_graph_of_launches():
    """Three refresh periods of 4 steps after 2 plain steps (t0 = 2): the
    persistent launch and the per-step graph give the same bits, with the
    near-conic problem's chains going through the overflow phase every step."""
    As, bs, Xs, nc = make_batch(3)
    got, st_p, info_p = run_batch(As, bs, Xs, nc, True, 14, t0=2)
    want, st_g, info_g = run_batch(As, bs, Xs, nc, False, 14, t0=2)
    assert info_p["graph_launches"] == 3 and info_g["graph_launches"] == 3
    np.testing.assert_array_equal(got, want)
    for key in ("steps", "rejections", "residual_rechecks", "tangent_fp64", "numeric_errors"):
        assert st_p[key] == st_g[key], key
    assert st_p["numeric_errors"] == 0
    # sort_keys counts the arcs (or merged bucket intervals) each chain's
    # sweep took: the overflow phase's 1024-thread CTA merges into 2048
    # buckets where the per-step CTA kernel (64 threads at m = 400) has 512,
    # so only its size is checked: the near-conic chains keep > 128 arcs each step
    assert st_p["sort_keys"] > 14 * 12 * 128 and st_g["sort_keys"] > 14 * 12 * 128


def test_persistent_long_arcs_equal_graph_of_launches():
    """Problems with rows of b_i <= 0 (arcs of at least a half circle, reduced
    to their union: the kernels' long-arc instantiations) batched with the
    ordinary ones: persistent launch and per-step graph give the same bits."""
    rng = np.random.default_rng(17)
    As, bs, Xs, nc = make_batch(19, with_cone=False)
    for kind, d, extra, n in (("orthant", 32, 0, 12), ("half", 48, 0, 9),
                              ("negative", 40, 40, 10)):
        A, b, X, _ = long_arc_instance(rng, d, n, kind, extra_rows=extra)
        As.append(A)
        bs.append(b)
        Xs.append(X)
        nc.append(n)
    got, st_p, _ = run_batch(As, bs, Xs, nc, True, 14, t0=2)
    want, st_g, _ = run_batch(As, bs, Xs, nc, False, 14, t0=2)
    np.testing.assert_array_equal(got, want)
    for key in ("steps", "rejections", "residual_rechecks", "tangent_fp64", "numeric_errors"):
        assert st_p[key] == st_g[key], key
    assert st_p["numeric_errors"] == 0


def test_persistent_repeated_calls_and_layout_change():
    """Two calls in a row (the period graph replayed from the cache), then a
    different chain layout (a new graph), each equal to the per-step graph."""
    As, bs, Xs, nc = make_batch(5, with_cone=False)
    for layout in (nc, [max(0, n - 3) for n in nc]):
        Xl = [X[:n] for X, n in zip(Xs, layout)]
        outs = []
        for persistent in (True, False):
            bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED, refresh_k=8)
            try:
                ess.ess_batch_set_persistent(bs_.batch, persistent)
                X = bs_.pack(Xl)
                bs_.run(layout, X, 16, seed=2, t0=0)
                bs_.run(layout, X, 16, seed=2, t0=16)
                outs.append(host(X))
            finally:
                bs_.close()
        np.testing.assert_array_equal(outs[0], outs[1])


def test_persistent_every_iterate_feasible():
    """Every recorded-free period leaves feasible states (FP64 check on the host)."""
    As, bs, Xs, nc = make_batch(7)
    got, st, _ = run_batch(As, bs, Xs, nc, True, 34, t0=2, refresh_k=8)
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED, refresh_k=8)
    try:
        parts = bs_.unpack(got, nc)
    finally:
        bs_.close()
    for p, (A, b) in enumerate(zip(As, bs)):
        if nc[p] == 0:
            continue
        assert (parts[p] @ A.T - b[None, :]).max() <= 0.0, f"problem {p}"
    assert st["numeric_errors"] == 0


def test_persistent_refused_for_fp64():
    As, bs, Xs, nc = make_batch(1, with_cone=False)
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_FP64, refresh_k=4)
    try:
        with pytest.raises(ess.EssError) as ei:
            ess.ess_batch_set_persistent(bs_.batch, True)
        assert ei.value.status == ess.ESS_ERR_UNSUPPORTED
        ess.ess_batch_set_persistent(bs_.batch, False)  # switching off is always allowed
    finally:
        bs_.close()


def test_dependency_wait_runs_out_and_the_batch_stays_usable():
    """A q dependency that nothing releases (ess_batch_selftest_wait raises
    every problem's target by one count): each chain step's wait gives up
    after the configured limit, the call returns ESS_ERR_TIMEOUT without a
    hang or a fault, and the same batch then runs periods equal to those of
    the per-step graph."""
    import time

    As, bs, Xs, nc = make_batch(9, with_cone=False)
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED, refresh_k=4,
                           wait_limit_us=20000)
    try:
        ess.ess_batch_set_persistent(bs_.batch, True)
        X = bs_.pack(Xs)
        t0 = time.perf_counter()
        with pytest.raises(ess.EssError) as e:
            ess.ess_batch_selftest_wait(bs_.batch, nc, X)
        assert e.value.status == ess.ESS_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        X = bs_.pack(Xs)
        before = ess.ess_batch_info(bs_.batch)["graph_launches"]
        bs_.run(nc, X, 10, seed=11, t0=2)
        got = host(X)
        assert ess.ess_batch_info(bs_.batch)["graph_launches"] - before == 2
    finally:
        bs_.close()
    want, _, _ = run_batch(As, bs, Xs, nc, False, 10, t0=2)
    np.testing.assert_array_equal(got, want)


def test_selftest_refused_without_the_persistent_launch():
    As, bs, Xs, nc = make_batch(1, with_cone=False)
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED, refresh_k=4)
    try:
        ess.ess_batch_set_persistent(bs_.batch, False)
        with pytest.raises(ess.EssError) as ei:
            ess.ess_batch_selftest_wait(bs_.batch, nc, bs_.pack(Xs))
        assert ei.value.status == ess.ESS_ERR_UNSUPPORTED
    finally:
        bs_.close()


def test_persistent_samples_follow_the_truncated_normal():
    """The persistent launch samples the target: a d = 1 interval [-0.5, 1.2]
    and a d = 2 box [-1, 3] x [-0.5, 1.2] (4096 chains each from 0) batched
    with an ordinary polytope, 64 steps at refresh_k = 16 (the last 48 in
    three persistent launches).  Each final state is one draw; KS tests
    against the exact truncated normals, and their means and variances
    (closed forms from scipy), hold within Monte Carlo error."""
    from scipy import stats

    rng = np.random.default_rng(41)
    A0, b0, X0 = feasible_instance(rng, 17, 60, 70, scale=1.0 / math.sqrt(17), slack=(0.1, 1.0))
    As = [np.array([[1.0], [-1.0]]), np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]]),
          A0]
    bs = [np.array([1.2, 0.5]), np.array([3.0, 1.0, 1.2, 0.5]), b0]
    n = 4096
    Xs = [np.zeros((n, 1)), np.zeros((n, 2)), X0]
    nc = [n, n, X0.shape[0]]
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED, refresh_k=16)
    try:
        ess.ess_batch_set_persistent(bs_.batch, True)
        X = bs_.pack(Xs)
        bs_.run(nc, X, 64, seed=5, t0=0)
        assert ess.ess_batch_info(bs_.batch)["graph_launches"] == 3
        parts = bs_.unpack(host(X), nc)
        st = bs_.stats()
    finally:
        bs_.close()
    assert st["numeric_errors"] == 0
    checks = [(parts[0][:, 0], stats.truncnorm(-0.5, 1.2)),
              (parts[1][:, 0], stats.truncnorm(-1.0, 3.0)),
              (parts[1][:, 1], stats.truncnorm(-0.5, 1.2))]
    for x, law in checks:
        assert stats.kstest(x, law.cdf).pvalue > 1e-3
        assert abs(x.mean() - law.mean()) < 5 * math.sqrt(law.var() / n)
        assert abs(x.var() - law.var()) < 0.1 * law.var()
    assert abs(np.corrcoef(parts[1][:, 0], parts[1][:, 1])[0, 1]) < 5 / math.sqrt(n)
    assert (parts[2] @ A0.T - b0[None, :]).max() <= 0.0
