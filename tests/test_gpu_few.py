"""ess_run_few: 1 to 16 FP64 chains, every step in one persistent kernel
(the paper's Sec. 4.2 single-chain and ten-chain experiments), against the
FP64 oracle's chains (Alg. 1 with the same Philox counters).

As in test_gpu_trajectories, runs are compared in segments of 8 steps: the
oracle restarts from the GPU's states and must land on the GPU's next states
within 1e-9 relative, chain by chain (differences in the last bits grow along
a trajectory).  Whole runs agree for most chains.  Sizes: the small config,
the Sec. 4.2 family (A d x d iid N(0, 1), b = A x0 + U[0, 1]) at d = 60 and
d = 300 with 1 and 10 chains, a probit-style orthant where every arc
survives the prune (the per-chain sort of 4096 arcs), d = 1.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
import workloads
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu

RTOL = 1e-9


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)), axis=1)


def _segments(A, b, X0, n_steps, seg, seed, refresh_k=32):
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_FP64, refresh_k=refresh_k)
    try:
        X = dev(X0)
        Xg = np.array(X0, dtype=np.float64)
        for t in range(0, n_steps, seg):
            want = oracle.run(A, b, Xg, seg, seed=seed, t0=t)[0]
            ess.ess_run_few(s.state, X, X.shape[0], t, seg, seed)
            Xg = host(X)
            gap = _rel(Xg, want)
            assert np.all(gap <= RTOL), (t + seg, float(gap.max()), int(np.argmax(gap)))
        st = s.stats()
    finally:
        s.close()
    assert np.max(Xg @ A.T - b) <= 0.0
    return st


def test_few_small_config_segments():
    inst = workloads.small(n_chains=16)
    st = _segments(inst.A, inst.b, inst.X0, 64, 8, 3)
    assert st["numeric_errors"] == 0 and st["steps"] == 16 * 64


@pytest.mark.parametrize("d,C", [(60, 1), (60, 10), (300, 1), (300, 10), (128, 16)])
def test_few_paper_family_segments(d, C):
    inst = workloads.paper_hd(d=d, n_chains=C, seed=d + C)
    _segments(inst.A, inst.b, inst.X0, 48, 8, 5)


def test_few_whole_run_and_generic_path():
    """A 96-step run (three refresh periods) against the oracle's 96 steps for
    most chains, and a short run equal to the generic FP64 path's."""
    inst = workloads.paper_hd(d=80, n_chains=12, seed=7)
    Xo, _, rej = oracle.run(inst.A, inst.b, inst.X0, 96, seed=9)
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64)
    try:
        X = dev(inst.X0)
        ess.ess_run_few(s.state, X, 12, 0, 96, 9)
        gap = _rel(host(X), Xo)
        assert np.mean(gap <= RTOL) >= 0.9, gap
        Xf = dev(inst.X0)
        ess.ess_run_few(s.state, Xf, 12, 0, 6, 4)
        Xr = dev(inst.X0)
        s.run(Xr, 6, seed=4)
        np.testing.assert_allclose(host(Xf), host(Xr), rtol=0, atol=1e-11)
    finally:
        s.close()


def test_few_all_arcs_survive():
    """b = 0 orthant (every arc has half-width pi / 2, none contains another):
    every row reaches the per-chain sort (4096 arcs for m = 4096)."""
    rng = np.random.default_rng(3)
    k = 4096
    L = np.tril(rng.standard_normal((k, k)) * 0.02) + np.eye(k)
    z = rng.standard_normal(k)
    f = L @ z
    A = -np.sign(f)[:, None] * L
    b = np.zeros(k)
    X0 = np.tile(z, (2, 1))
    _segments(A, b, X0, 4, 2, 11)


def test_few_interval_d1():
    inst = workloads.interval(-0.5, 1.2, n_chains=16)
    _segments(inst.A, inst.b, inst.X0, 40, 8, 2)


def test_few_records_and_final_state():
    import torch
    inst = workloads.paper_hd(d=40, n_chains=3, seed=1)
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64)
    try:
        X = dev(inst.X0)
        S = torch.zeros((3, 5, 40), dtype=torch.float64, device="cuda")
        ess.ess_run_few(s.state, X, 3, 0, 10, 8, S, 2)
        S, Xg = host(S), host(X)
    finally:
        s.close()
    np.testing.assert_array_equal(S[:, 4], Xg)
    want = [oracle.run(inst.A, inst.b, inst.X0, 2 * (r + 1), seed=8)[0] for r in range(5)]
    for r in range(5):
        gap = _rel(S[:, r], want[r])
        assert np.all(gap <= RTOL), (r, gap)


def test_few_errors():
    inst = workloads.paper_hd(d=20, n_chains=2, seed=2)
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64)
    try:
        bad = inst.X0.copy()
        bad[1] += 10.0 * inst.A[0] / np.linalg.norm(inst.A[0])
        assert np.max(bad[1] @ inst.A.T - inst.b) > 0
        X = dev(bad)
        with pytest.raises(ess.EssError) as e:
            ess.ess_run_few(s.state, X, 2, 0, 5, 1)
        assert e.value.status == ess.ESS_ERR_INFEASIBLE_X0
        np.testing.assert_array_equal(host(X), bad)
        X17 = dev(np.tile(inst.X0[0], (17, 1)))
        with pytest.raises(ess.EssError) as e:
            ess.ess_run_few(s.state, X17, 17, 0, 5, 1)
        assert e.value.status == ess.ESS_ERR_ARG
    finally:
        s.close()
    sm = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_MIXED)
    try:
        with pytest.raises(ess.EssError) as e:
            ess.ess_run_few(sm.state, dev(inst.X0), 2, 0, 5, 1)
        assert e.value.status == ess.ESS_ERR_UNSUPPORTED
    finally:
        sm.close()
