"""Batched problems (ess_batch_*): polytopes of uneven d, m and chain counts
advanced together, against the FP64 oracle run problem by problem.

The batch only changes the work layout (packed states, grouped GEMM work
items, per-chain problem views, graph replays); every chain must follow the
one-problem sampler of Alg. 1 with the problem index in its Philox counter.
Sizes cross the 64-row and 64-chain work-item tiles and the 16-wide K chunk,
and include d = 1 and a problem with no chains.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
import workloads
from gpu_helpers import dev, host, oracle_steps, feasible_instance, fp16x3_bound, grid_instance, \
    long_arc_instance, mixed_endpoint_bounds, mixed_exempt

pytestmark = pytest.mark.gpu

# (d, m, chains)
SPECS = [(1, 2, 3), (3, 5, 4), (10, 20, 16), (17, 60, 70), (40, 130, 9), (64, 64, 0),
         (33, 100, 65)]


def make_batch(seed, specs=SPECS):
    rng = np.random.default_rng(seed)
    As, bs, Xs = [], [], []
    for d, m, n in specs:
        A, b, X = feasible_instance(rng, d, m, max(n, 1), scale=1.0 / math.sqrt(d),
                                    slack=(0.1, 1.0))
        As.append(A)
        bs.append(b)
        Xs.append(X[:n])
    return As, bs, Xs, [n for _, _, n in specs]


def test_batch_fp64_run_reproduces_oracle():
    """20 steps with refresh_k = 8: direct steps, one graph-replayed period,
    direct steps again; every problem's chains equal the oracle's."""
    As, bs, Xs, nc = make_batch(1)
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_FP64, refresh_k=8)
    try:
        X = bs_.pack(Xs)
        bs_.run(nc, X, 20, seed=9)
        got = bs_.unpack(X, nc)
        info = ess.ess_batch_info(bs_.batch)
        st = bs_.stats()
    finally:
        bs_.close()
    assert info["graph_launches"] == 1
    for p, (A, b, X0) in enumerate(zip(As, bs, Xs)):
        if X0.shape[0] == 0:
            continue
        want, _, rej = oracle.run(A, b, X0, 20, seed=9, problem=p)
        np.testing.assert_allclose(got[p], want, rtol=0, atol=1e-8, err_msg=f"problem {p}")
    assert st["numeric_errors"] == 0
    assert st["steps"] == sum(nc) * 20


@pytest.mark.parametrize("form", [ess.ESS_PREC_FP64, ess.ESS_PREC_MIXED])
def test_batch_graph_replay_is_bit_identical(form):
    """Graph replays and plain launches give the same bits."""
    As, bs, Xs, nc = make_batch(2)
    out = []
    for graphs in (True, False):
        bs_ = ess.BatchSampler(As, bs, precision=form, refresh_k=4)
        try:
            ess.ess_batch_set_graphs(bs_.batch, graphs)
            X = bs_.pack(Xs)
            bs_.run(nc, X, 22, seed=4, t0=2)
            out.append(host(X))
            info = ess.ess_batch_info(bs_.batch)
        finally:
            bs_.close()
        assert info["graph_launches"] == (5 if graphs else 0)
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("form", [ess.ESS_PREC_FP64, ess.ESS_PREC_MIXED])
def test_batch_draws_ahead_are_bit_identical(form):
    """nu of step t + 1 drawn on a side stream beside step t (plain launches
    and graph replays) gives the bits of strictly sequential launches
    (per-phase timing on), with a layout change between runs (the second
    runs swap which nu buffers and operand maps are current)."""
    As, bs, Xs, nc = make_batch(3)
    nc2 = [max(0, n - 3) for n in nc]
    out = []
    for timing, graphs in ((True, False), (False, False), (False, True)):
        bs_ = ess.BatchSampler(As, bs, precision=form, refresh_k=4)
        try:
            ess.ess_batch_set_graphs(bs_.batch, graphs)
            ess.ess_batch_set_timing(bs_.batch, timing)
            X = bs_.pack(Xs)
            bs_.run(nc, X, 19, seed=6, t0=1)
            X2 = bs_.pack([x[:n] for x, n in zip(Xs, nc2)])
            bs_.run(nc2, X2, 13, seed=6, t0=3)
            out.append((host(X), host(X2)))
        finally:
            bs_.close()
    for o in out[1:]:
        np.testing.assert_array_equal(out[0][0], o[0])
        np.testing.assert_array_equal(out[0][1], o[1])


def test_batch_fp64_step_with_draws():
    """One step with given draws: theta within 1e-10 rad, x' within 1e-9
    relative of the oracle's one-step map, for every chain of every problem."""
    As, bs, Xs, nc = make_batch(3)
    rng = np.random.default_rng(5)
    NUs = [rng.standard_normal(X.shape) for X in Xs]
    U = rng.uniform(size=sum(nc))
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_FP64)
    try:
        Xn, th, rej = bs_.step_with_draws(nc, bs_.pack(Xs), bs_.pack(NUs), dev(U))
        Xn = bs_.unpack(Xn, nc)
        th, rej = host(th), host(rej)
    finally:
        bs_.close()
    at = 0
    for p, (A, b, X, NU) in enumerate(zip(As, bs, Xs, NUs)):
        ref = oracle_steps(A, b, X, NU, U[at:at + X.shape[0]])
        for c, r in enumerate(ref):
            assert abs(th[at + c] - r.theta) <= 1e-10, (p, c, th[at + c], r.theta)
            assert bool(rej[at + c]) == r.rejected
            scale = np.maximum(1.0, np.abs(r.x_next))
            assert np.all(np.abs(Xn[p][c] - r.x_next) <= 1e-9 * scale), (p, c)
        at += X.shape[0]


def test_batch_mixed_step_with_draws():
    """Mixed form, one step with given draws, on grid inputs (exact P and Q):
    theta within 1e-5 rad and x' within 1e-5 relative of the oracle's one-step
    map for every chain not exempted by the a-priori conditioning bound of its
    arc endpoints (gpu_helpers.mixed_exempt); zero infeasible iterates."""
    rng = np.random.default_rng(6)
    As, bs, Xs, NUs = [], [], [], []
    for d, m, n in SPECS:
        A, b, X, NU = grid_instance(rng, d, m, max(n, 1), scale=1.0 / math.sqrt(d),
                                    slack=(0.1, 1.0))
        As.append(A)
        bs.append(b)
        Xs.append(X[:n])
        NUs.append(NU[:n])
    nc = [n for _, _, n in SPECS]
    U = rng.uniform(size=sum(nc))
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED)
    try:
        Xn, th, rej = bs_.step_with_draws(nc, bs_.pack(Xs), bs_.pack(NUs), dev(U))
        Xn = bs_.unpack(Xn, nc)
        th, rej = host(th), host(rej)
    finally:
        bs_.close()
    at, exempt_total, total = 0, 0, 0
    for p, (A, b, X, NU) in enumerate(zip(As, bs, Xs, NUs)):
        if X.shape[0]:
            assert np.max(Xn[p] @ A.T - b) <= 0.0, p
        ref = oracle_steps(A, b, X, NU, U[at:at + X.shape[0]])
        amp, arith = mixed_endpoint_bounds(A, b, X, NU)
        exempt = mixed_exempt(ref, amp, arith, 0.5e-5)
        for c, r in enumerate(ref):
            total += 1
            if exempt[c]:
                exempt_total += 1
                continue
            assert abs(th[at + c] - r.theta) <= 1e-5, (p, c, th[at + c], r.theta)
            if rej[at + c]:
                np.testing.assert_array_equal(Xn[p][c], X[c])
            else:
                scale = (1.0 + np.abs(r.x_next)) * (1.0 + np.abs(NU[c]))
                assert np.all(np.abs(Xn[p][c] - r.x_next) <= 1e-5 * scale), (p, c)
        at += X.shape[0]
    assert exempt_total <= 0.05 * total, (exempt_total, total)


# problems with rows of b_i <= 0 (kind, d, extra rows, chains), beside one without
LONG_SPECS = [("orthant", 32, 0, 12), ("half", 48, 0, 9), ("negative", 40, 40, 10)]


def make_long_batch(seed, grid=False):
    rng = np.random.default_rng(seed)
    if grid:
        A, b, X, NU = grid_instance(rng, 10, 20, 16, scale=1.0 / math.sqrt(10), slack=(0.1, 1.0))
    else:
        A, b, X = feasible_instance(rng, 10, 20, 16, scale=1.0 / math.sqrt(10), slack=(0.1, 1.0))
        NU = rng.standard_normal(X.shape)
    As, bs, Xs, NUs = [A], [b], [X], [NU]
    for kind, d, extra, n in LONG_SPECS:
        A, b, X, NU = long_arc_instance(rng, d, n, kind, extra_rows=extra, grid=grid)
        As.append(A)
        bs.append(b)
        Xs.append(X)
        NUs.append(NU)
    return As, bs, Xs, NUs, [X.shape[0] for X in Xs]


def test_batch_long_arcs_fp64_run_reproduces_oracle():
    """Problems whose rows with b_i <= 0 give arcs of at least a half circle
    (an orthant, one with short arcs between, one with b_i < 0 and extra
    rows) batched with an ordinary polytope: 20 steps with refresh_k = 8, every
    chain equal to the oracle's (the batch kernels drop the arcs inside the
    union of the long arcs, which leaves I_act as it is)."""
    As, bs, Xs, _, nc = make_long_batch(21)
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_FP64, refresh_k=8)
    try:
        X = bs_.pack(Xs)
        bs_.run(nc, X, 20, seed=4)
        got = bs_.unpack(X, nc)
        st = bs_.stats()
    finally:
        bs_.close()
    for p, (A, b, X0) in enumerate(zip(As, bs, Xs)):
        want, _, _ = oracle.run(A, b, X0, 20, seed=4, problem=p)
        np.testing.assert_allclose(got[p], want, rtol=0, atol=1e-8, err_msg=f"problem {p}")
    assert st["numeric_errors"] == 0


def test_batch_long_arcs_mixed_step_with_draws():
    """The same problems in the mixed form on grid inputs, one step with given
    draws: theta within 1e-5 rad and x' within 1e-5 relative of the oracle's
    for every chain not exempted by the a-priori bound of its arc endpoints;
    no infeasible iterate."""
    As, bs, Xs, NUs, nc = make_long_batch(22, grid=True)
    rng = np.random.default_rng(23)
    U = rng.uniform(size=sum(nc))
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED)
    try:
        Xn, th, rej = bs_.step_with_draws(nc, bs_.pack(Xs), bs_.pack(NUs), dev(U))
        Xn = bs_.unpack(Xn, nc)
        th, rej = host(th), host(rej)
    finally:
        bs_.close()
    at, exempt_total, total = 0, 0, 0
    for p, (A, b, X, NU) in enumerate(zip(As, bs, Xs, NUs)):
        assert np.max(Xn[p] @ A.T - b) <= 0.0, p
        ref = oracle_steps(A, b, X, NU, U[at:at + X.shape[0]])
        amp, arith = mixed_endpoint_bounds(A, b, X, NU)
        exempt = mixed_exempt(ref, amp, arith, 0.5e-5)
        for c, r in enumerate(ref):
            total += 1
            if exempt[c]:
                exempt_total += 1
                continue
            assert abs(th[at + c] - r.theta) <= 1e-5, (p, c, th[at + c], r.theta)
            if rej[at + c]:
                np.testing.assert_array_equal(Xn[p][c], X[c])
            else:
                scale = (1.0 + np.abs(r.x_next)) * (1.0 + np.abs(NU[c]))
                assert np.all(np.abs(Xn[p][c] - r.x_next) <= 1e-5 * scale), (p, c)
        at += X.shape[0]
    assert exempt_total <= 0.05 * total, (exempt_total, total)


@pytest.mark.parametrize("form", [ess.ESS_PREC_FP64, ess.ESS_PREC_MIXED])
def test_batch_products(form):
    """P = A x (refresh path, FP64-class in both forms) and Q = A nu (the
    tensor-core FP16x3 products in the mixed form, within their bound)."""
    As, bs, Xs, nc = make_batch(8)
    rng = np.random.default_rng(9)
    NUs = [rng.standard_normal(X.shape) for X in Xs]
    bs_ = ess.BatchSampler(As, bs, precision=form)
    try:
        P, Q = bs_.products(nc, bs_.pack(Xs), bs_.pack(NUs))
        P, Q = bs_.unpack(P, nc, "m"), bs_.unpack(Q, nc, "m")
    finally:
        bs_.close()
    for p, (A, X, NU) in enumerate(zip(As, Xs, NUs)):
        if form == ess.ESS_PREC_MIXED:
            X = np.asarray(X, np.float32).astype(np.float64)
            NU = np.asarray(NU, np.float32).astype(np.float64)
            A32 = np.asarray(A, np.float32).astype(np.float64)
            qtol = fp16x3_bound(A32, NU)
            np.testing.assert_array_less(np.abs(Q[p] - NU @ A32.T), qtol + 1e-300)
            # a wrong operand layout would not stay far inside the bound
            if Q[p].size:
                assert np.median(np.abs(Q[p] - NU @ A32.T) / (qtol + 1e-300)) < 0.2
        else:
            np.testing.assert_allclose(Q[p], NU @ A.T, rtol=0,
                                       atol=1e-13 * (1 + np.abs(NU).sum()))
        ptol = 1e-12 * (np.abs(X) @ np.abs(A).T) + 1e-300
        np.testing.assert_array_less(np.abs(P[p] - X @ A.T), ptol)


@pytest.mark.parametrize("form", [ess.ESS_PREC_FP64, ess.ESS_PREC_MIXED])
def test_batch_every_iterate_feasible(form):
    """The uneven-batch workload (reduced): every recorded iterate of every
    chain satisfies its polytope in FP64."""
    import torch
    insts = workloads.batched(seed=3, n_problems=24, n_iter=40, d_range=(8, 96),
                              c_range=(1, 40))
    As = [i.A for i in insts]
    bs = [i.b for i in insts]
    nc = [i.X0.shape[0] for i in insts]
    bs_ = ess.BatchSampler(As, bs, precision=form, refresh_k=8)
    try:
        X = bs_.pack([i.X0 for i in insts])
        tx = X.numel()
        S = torch.zeros((40, tx), dtype=bs_.sample_dtype, device="cuda")
        bs_.run(nc, X, 40, seed=2, samples=S, record_every=1)
        S = host(S).astype(np.float64)
        st = bs_.stats()
    finally:
        bs_.close()
    for r in range(40):
        rows = bs_.unpack(S[r], nc)
        for p, inst in enumerate(insts):
            assert np.max(rows[p] @ inst.A.T - inst.b) <= 0.0, (r, p)
    assert st["numeric_errors"] == 0


def test_batch_infeasible_start_is_refused():
    As, bs, Xs, nc = make_batch(10)
    Xs = [X.copy() for X in Xs]
    Xs[2][3] = 1e3  # far outside problem 2
    bs_ = ess.BatchSampler(As, bs, precision=ess.ESS_PREC_MIXED)
    try:
        with pytest.raises(ess.EssError):
            bs_.run(nc, bs_.pack(Xs), 5, seed=0)
    finally:
        bs_.close()
