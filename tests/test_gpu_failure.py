"""Error paths of the step that need no GPU fault: non-finite directions.

A caller-supplied nu with NaN or Inf makes q = A nu non-finite for that chain
only.  The chain kernels then reject the move (Sec. 3.3: the chain stays at
x_t), count a numeric error, and the call returns ESS_ERR_NUMERIC.  Every
other chain must still take the oracle's step, and the state must stay usable.
"""
import math

import numpy as np
import pytest

import paper_2407_10449_gb300 as ess
from gpu_helpers import dev, host, grid_instance, oracle_steps, f32

pytestmark = pytest.mark.gpu

FORMS = [("fp64", ess.ESS_PREC_FP64, {}),
         ("fp64_split", ess.ESS_PREC_FP64, {"fp64_products": ess.ESS_PRODUCTS_SPLIT}),
         ("mixed", ess.ESS_PREC_MIXED, {})]


@pytest.mark.parametrize("name,prec,cfg", FORMS, ids=[f[0] for f in FORMS])
def test_non_finite_nu_rejects_and_reports(name, prec, cfg):
    import torch
    rng = np.random.default_rng(41)
    d, m, n = 16, 40, 24
    A, b, X, NU = grid_instance(rng, d, m, n, scale=1.0 / math.sqrt(d), slack=(0.1, 0.8))
    U = rng.uniform(size=n)
    bad = {3: np.nan, 5: np.inf, 11: -np.inf}
    NUb = NU.copy()
    for c, v in bad.items():
        NUb[c, c % d] = v
    if prec == ess.ESS_PREC_MIXED:
        X, NU, NUb = f32(X), f32(NU), f32(NUb)
    s = ess.Sampler(A, b, precision=prec, **cfg)
    try:
        Xd = dev(X)
        Xn = torch.empty_like(Xd)
        th = torch.empty(n, dtype=torch.float64, device="cuda")
        rej = torch.empty(n, dtype=torch.int32, device="cuda")
        npc = torch.empty(n, dtype=torch.int32, device="cuda")
        with pytest.raises(ess.EssError) as e:
            ess.ess_step_with_draws(s.state, Xd, dev(NUb), dev(U), n, Xn, th, None, 0, npc,
                                    rej, None)
        assert e.value.status == ess.ESS_ERR_NUMERIC
        Xn, th, rej = host(Xn), host(th), host(rej)
        st = s.stats()
        assert st["numeric_errors"] == len(bad)
        good = [c for c in range(n) if c not in bad]
        for c in bad:
            assert rej[c] == 1
            np.testing.assert_array_equal(Xn[c], X[c])
        refs = oracle_steps(A, b, X[good], NU[good], U[good])
        tol = 1e-10 if prec == ess.ESS_PREC_FP64 else 1e-5
        for c, r in zip(good, refs):
            assert abs(th[c] - r.theta) <= tol, (c, th[c], r.theta)
            assert np.all(np.abs(Xn[c] - r.x_next) <= 10 * tol * (1 + np.abs(r.x_next)))
        # the state is still usable: the same step with finite draws succeeds
        Xn2, th2, _, _, _ = s.step_with_draws(Xd, dev(NU), dev(U))
        refs = oracle_steps(A, b, X, NU, U)
        assert max(abs(float(t) - r.theta) for t, r in zip(host(th2), refs)) <= tol
    finally:
        s.close()


def test_bounded_wait_runs_out_and_the_device_stays_usable():
    """A grid barrier of the persistent few-chain kernel whose dependency is
    never released (one CTA withholds its arrival) gives up after the
    configured limit: the call returns ESS_ERR_TIMEOUT, nothing hangs or
    faults, and the same state then runs the oracle's chains."""
    import time

    import oracle
    import workloads
    inst = workloads.paper_hd(d=64, n_chains=3, seed=3)
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64, wait_limit_us=20000)
    try:
        t0 = time.perf_counter()
        with pytest.raises(ess.EssError) as e:
            ess.ess_selftest_wait(s.state)
        assert e.value.status == ess.ESS_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 10.0
        X = dev(inst.X0)
        ess.ess_run_few(s.state, X, 3, 0, 6, 2)
        want = oracle.run(inst.A, inst.b, inst.X0, 6, seed=2)[0]
        np.testing.assert_allclose(host(X), want, rtol=0, atol=1e-9 * (1 + np.abs(want).max()))
    finally:
        s.close()
    with pytest.raises(ess.EssError):
        ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64, wait_limit_us=-1)
