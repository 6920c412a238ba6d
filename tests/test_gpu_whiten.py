"""App. A on the GPU: x = L u + mu for batches of samples (ess_whitener_*).

* FP64 samples: FP64 FMAs, within a few ulps of the oracle's x = L u + mu.
* float samples: the scaled FP16x3 tensor-core GEMM, within its stated bound
  (16 + d/16) 2^-24 sum_j |L_ij||u_j| plus the FP32 rounding of the result.
* A run in whitened coordinates (App. A) mapped back on the GPU satisfies the
  original constraints.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
import workloads
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


def random_chol(rng, d):
    M = rng.standard_normal((d, d)) / math.sqrt(d)
    K = M @ M.T + 0.1 * np.eye(d)
    return np.linalg.cholesky(K)


@pytest.mark.parametrize("d,n,with_mu", [(1, 5, True), (50, 130, False), (300, 257, True),
                                         (1000, 64, True)])
def test_whitener_fp64(d, n, with_mu):
    import torch
    rng = np.random.default_rng(d + n)
    L = random_chol(rng, d)
    mu = rng.standard_normal(d) if with_mu else None
    U = rng.standard_normal((n, d))
    w = ess.Whitener(L, mu)
    try:
        X = host(w(dev(U)))
    finally:
        w.close()
    want = oracle.unwhiten(L, mu, U)
    tol = 1e-13 * (np.abs(U) @ np.abs(L).T + (np.abs(mu) if mu is not None else 0.0)) + 1e-300
    assert np.all(np.abs(X - want) <= tol)


@pytest.mark.parametrize("d,n,with_mu", [(3, 7, True), (137, 300, True), (1000, 130, False),
                                         (2000, 128, True)])
def test_whitener_fp16x3(d, n, with_mu):
    import torch
    rng = np.random.default_rng(3 * d + n)
    L = random_chol(rng, d)
    mu = rng.standard_normal(d) if with_mu else None
    U = rng.standard_normal((n, d)).astype(np.float32)
    w = ess.Whitener(L, mu)
    try:
        X = host(w(dev(U, torch.float32))).astype(np.float64)
    finally:
        w.close()
    U64 = U.astype(np.float64)
    L32 = L.astype(np.float32).astype(np.float64)
    prod = U64 @ L32.T
    want = prod + (mu if mu is not None else 0.0)
    bound = (16 + d / 16) * 2.0**-24 * (np.abs(U64) @ np.abs(L32).T)
    # L rounded to float, the product rounded to float, + mu rounded
    tol = (bound + 2.0**-24 * (np.abs(U64) @ np.abs(L).T) + 2.0**-23 * (np.abs(prod) +
           (np.abs(mu) if mu is not None else 0.0)) + 1e-30)
    err = np.abs(X - want)
    assert np.all(err <= tol), float((err / tol).max())


@pytest.mark.parametrize("form", [ess.ESS_PREC_FP64, ess.ESS_PREC_MIXED])
def test_probit_run_mapped_back_is_feasible(form):
    """Config-4-style probit orthant (n = 120 points): sample u under
    (A0 L) u <= 0 and map the recorded samples x = L u on the GPU; every x must
    satisfy y_i x_i >= 0 (A0 x <= 0) up to the map's rounding."""
    import torch
    pb = workloads.probit(n=120, n_chains=64)
    A, b = ess.ess_whiten(pb["A0"], pb["b"], pb["mu"], pb["L"])
    s = ess.Sampler(A, b, precision=form)
    w = ess.Whitener(pb["L"], pb["mu"])
    try:
        X = dev(pb["X0"])
        S = torch.zeros((64, 30, 120), dtype=s.sample_dtype, device="cuda")
        s.run(X, 30, seed=1, samples=S, record_every=1)
        Xs = host(w(S.reshape(-1, 120))).astype(np.float64)
        Uh = host(S).reshape(-1, 120).astype(np.float64)
    finally:
        w.close()
        s.close()
    viol = Xs @ pb["A0"].T - pb["b"]
    # the map's error bound per row of L
    d = 120
    eps = (16 + d / 16 + 4) * 2.0**-24 if form == ess.ESS_PREC_MIXED else 1e-13
    scale = np.abs(Uh) @ np.abs(pb["L"]).T
    assert np.all(viol <= eps * scale + 1e-300)
    # and the samples themselves are exactly feasible in whitened coordinates
    assert np.max(Uh @ A.T - b) <= 0.0
