"""ess_step_noalloc: the FP64 chain step for callers that may not allocate.

Some callers cannot call cudaMalloc when they want a step (a host framework
that owns the device-memory budget, an allocation-free request path, a thread
whose stream is being captured).  The entry point takes every buffer from the
caller and its scratch from a fixed array inside the library.  This test calls
it through the C ABI twice in a row (the second call reuses the scratch left by
the first) and checks each result against ess_step_with_draws, the existing
entry point of the same map, at the FP64 tolerances of the parity tests.
It lives in its own file, collected last.
"""
import numpy as np
import pytest

import paper_2407_10449_gb300 as ess
from gpu_helpers import dev, host, feasible_instance

pytestmark = pytest.mark.gpu

ANG_TOL = 1e-10
X_RTOL = 1e-9


def _reference(A, b, X, NU, U):
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_FP64)
    try:
        Xn, th, _, _, rej = s.step_with_draws(dev(X), dev(NU), dev(U))
        return host(Xn), host(th), host(rej)
    finally:
        s.close()


def _noalloc(A, b, X, NU, U):
    import torch
    n, d = X.shape
    Xn = torch.empty((n, d), dtype=torch.float64, device="cuda")
    th = torch.empty(n, dtype=torch.float64, device="cuda")
    rej = torch.empty(n, dtype=torch.int32, device="cuda")
    ess.ess_step_noalloc(dev(A), dev(b), dev(X), dev(NU), dev(U), Xn, th, rej)
    return host(Xn), host(th), host(rej)


def _same(got, want):
    Xg, tg, rg = got
    Xw, tw, rw = want
    assert np.all(np.abs(tg - tw) <= ANG_TOL)
    assert np.array_equal(rg, rw)
    assert np.all(np.abs(Xg - Xw) <= X_RTOL * np.maximum(1.0, np.abs(Xw)))


def test_noalloc_matches_step_with_draws_twice():
    rng = np.random.default_rng(77)
    d, m, n = 45, 301, 97
    A, b, X = feasible_instance(rng, d, m, n)
    NU1, U1 = rng.standard_normal((n, d)), rng.uniform(size=n)
    first = _noalloc(A, b, X, NU1, U1)
    _same(first, _reference(A, b, X, NU1, U1))
    # second call in a row, starting from the first call's output
    X2 = first[0]
    NU2, U2 = rng.standard_normal((n, d)), rng.uniform(size=n)
    second = _noalloc(A, b, X2, NU2, U2)
    _same(second, _reference(A, b, X2, NU2, U2))
    assert np.max(second[0] @ A.T - b) <= 0.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    d, m = 4, 2000
    n = ess.NOALLOC_SCRATCH_BYTES // (16 * m) + 1   # P and Q no longer fit
    A = torch.zeros((m, d), dtype=torch.float64, device="cuda")
    b = torch.ones(m, dtype=torch.float64, device="cuda")
    X = torch.zeros((n, d), dtype=torch.float64, device="cuda")
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(ess.EssError) as e:
        ess.ess_step_noalloc(A, b, X, X, u, torch.empty_like(X))
    assert e.value.status == ess.ESS_ERR_ARG
    assert "16 MiB" in str(e.value)
