"""ess_step_noalloc: the FP64 chain step for callers that may not allocate.

Some callers cannot call cudaMalloc when they want a step: a plugin inside a
host framework that owns the device-memory budget, or a request path that must
stay off the allocator and its implicit synchronization.  The entry point takes
every buffer from the caller and its scratch from a fixed array inside the
library.  These tests call it through the C ABI and check its results against
the FP64 oracle's one-step map (Alg. 1 with given nu and u) at the FP64
tolerances of the parity tests: two calls in a row (the second reuses the
scratch left by the first), the 1024-thread CTA path (m near 8192), NULL
optional outputs on a side stream, and the error paths (an infeasible start,
sizes beyond the scratch, a d too large for shared memory).  The file is
collected last.
"""
import numpy as np
import pytest

import paper_2407_10449_gb300 as ess
from gpu_helpers import dev, host, feasible_instance, oracle_steps

pytestmark = pytest.mark.gpu

ANG_TOL = 1e-10
X_RTOL = 1e-9


def _noalloc(A, b, X, NU, U, outputs=True, stream=None):
    import torch
    n, d = X.shape
    Xn = torch.empty((n, d), dtype=torch.float64, device="cuda")
    th = torch.empty(n, dtype=torch.float64, device="cuda") if outputs else None
    rej = torch.empty(n, dtype=torch.int32, device="cuda") if outputs else None
    ess.ess_step_noalloc(dev(A), dev(b), dev(X), dev(NU), dev(U), Xn, th, rej, stream=stream)
    return host(Xn), None if th is None else host(th), None if rej is None else host(rej)


def _check_against_oracle(got, A, b, X, NU, U):
    Xg, tg, rg = got
    want = oracle_steps(A, b, X, NU, U)
    Xw = np.stack([r.x_next for r in want])
    assert np.all(np.abs(Xg - Xw) <= X_RTOL * np.maximum(1.0, np.abs(Xw)))
    if tg is not None:
        tw = np.array([r.theta for r in want])
        assert np.all(np.abs(tg - tw) <= ANG_TOL)
    if rg is not None:
        rw = np.array([int(r.rejected) for r in want])
        assert np.array_equal(rg, rw)


def test_noalloc_matches_oracle_twice():
    rng = np.random.default_rng(77)
    d, m, n = 45, 301, 97
    A, b, X = feasible_instance(rng, d, m, n)
    NU1, U1 = rng.standard_normal((n, d)), rng.uniform(size=n)
    first = _noalloc(A, b, X, NU1, U1)
    _check_against_oracle(first, A, b, X, NU1, U1)
    # second call in a row, starting from the first call's output
    X2 = first[0]
    NU2, U2 = rng.standard_normal((n, d)), rng.uniform(size=n)
    second = _noalloc(A, b, X2, NU2, U2)
    _check_against_oracle(second, A, b, X2, NU2, U2)
    assert np.max(second[0] @ A.T - b) <= 0.0


def test_noalloc_large_m_cta_path():
    """m = 8000 takes the 1024-thread CTA kernel."""
    rng = np.random.default_rng(78)
    d, m, n = 12, 8000, 3
    A, b, X = feasible_instance(rng, d, m, n)
    NU, U = rng.standard_normal((n, d)), rng.uniform(size=n)
    _check_against_oracle(_noalloc(A, b, X, NU, U), A, b, X, NU, U)


def test_noalloc_null_outputs_side_stream():
    import torch
    rng = np.random.default_rng(79)
    d, m, n = 30, 150, 40
    A, b, X = feasible_instance(rng, d, m, n)
    NU, U = rng.standard_normal((n, d)), rng.uniform(size=n)
    side = torch.cuda.Stream()
    got = _noalloc(A, b, X, NU, U, outputs=False, stream=side)
    _check_against_oracle(got, A, b, X, NU, U)


def test_noalloc_infeasible_start_leaves_outputs():
    import torch
    rng = np.random.default_rng(80)
    d, m, n = 8, 40, 5
    A, b, X = feasible_instance(rng, d, m, n)
    X[2] = 10.0 * A[0] / np.linalg.norm(A[0]) + X[2]  # pushes chain 2 out
    assert np.max(X[2] @ A.T - b) > 0.0
    NU, U = rng.standard_normal((n, d)), rng.uniform(size=n)
    Xn = torch.full((n, d), 7.0, dtype=torch.float64, device="cuda")
    th = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(ess.EssError) as e:
        ess.ess_step_noalloc(dev(A), dev(b), dev(X), dev(NU), dev(U), Xn, th)
    assert e.value.status == ess.ESS_ERR_INFEASIBLE_X0
    assert torch.all(Xn == 7.0) and torch.all(th == 7.0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    d, m = 4, 2000

    def r(v):
        return -(-v // 256) * 256

    n = 1
    while 512 + r(8 * m) + 2 * r(8 * (n + 1) * m) <= ess.NOALLOC_SCRATCH_BYTES:
        n += 1
    n += 1  # the first chain count that no longer fits
    A = torch.zeros((m, d), dtype=torch.float64, device="cuda")
    b = torch.ones(m, dtype=torch.float64, device="cuda")
    X = torch.zeros((n, d), dtype=torch.float64, device="cuda")
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(ess.EssError) as e:
        ess.ess_step_noalloc(A, b, X, X, u, torch.empty_like(X))
    assert e.value.status == ess.ESS_ERR_ARG
    assert "16 MiB" in str(e.value)


def test_noalloc_rejects_d_beyond_shared_memory():
    import torch
    d, m = 8000, 8192
    A = torch.zeros((m, d), dtype=torch.float64, device="cuda")
    b = torch.ones(m, dtype=torch.float64, device="cuda")
    X = torch.zeros((1, d), dtype=torch.float64, device="cuda")
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ess.EssError) as e:
        ess.ess_step_noalloc(A, b, X, X, u, torch.empty_like(X))
    assert e.value.status == ess.ESS_ERR_UNSUPPORTED


def test_noalloc_wrapper_refuses_bad_tensors():
    import torch
    A = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    b = torch.ones(10, dtype=torch.float64, device="cuda")
    X = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    u = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ess.ess_step_noalloc(A, b, X.float(), X, u, torch.empty_like(X))
    with pytest.raises(ValueError):
        ess.ess_step_noalloc(A, b, X, torch.zeros((4, 2), dtype=torch.float64, device="cuda"),
                             u, torch.empty_like(X))
    with pytest.raises(ValueError):
        ess.ess_step_noalloc(A, b, X, X, u[:3], torch.empty_like(X))
    with pytest.raises(ValueError):
        ess.ess_step_noalloc(A, b, X, X, u, torch.empty_like(X),
                             rejected=torch.zeros(4, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        ess.ess_step_noalloc(A, b, X.cpu(), X, u, torch.empty_like(X))
    with pytest.raises(ValueError):
        ess.ess_step_noalloc(A, b, torch.zeros((3, 4), dtype=torch.float64,
                                               device="cuda").t(), X, u, torch.empty_like(X))
