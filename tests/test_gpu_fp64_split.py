"""FP64 form with its products q = A nu and p = A x from exact fixed-point
splits on the tensor cores (ess_config.fp64_products = ESS_PRODUCTS_SPLIT).

The products must stay within the split's stated bound of the exact values:
d (3 + K(K-1)/2) 2^-(wK) s_i t_c from the truncated 56-bit slices (w-bit
integer slices, K = ceil(56 / w), s_i and t_c the power-of-two row scales just
above max |a_i| and max |x_c|), plus N^2 2^-48 sum_j |a_ij x_j| from the
(hi, lo) float pairs the N = K(K+1)/2 slice products are summed into (each
addition exact, the low parts summed in float), plus the final rounding.  With products
that accurate the one-step map must meet the FP64 form's bar against the
oracle (endpoints and theta within 1e-10 rad, x' within 1e-9 relative, same
rejections), runs must reproduce the oracle's chains, and infeasible starts
must still be refused.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
import workloads
from gpu_helpers import dev, host, feasible_instance
from test_gpu_fp64_step import check_fp64

pytestmark = pytest.mark.gpu

SPLIT = dict(fp64_products=ess.ESS_PRODUCTS_SPLIT)


def split_bound(A, X, bits=56):
    d = A.shape[1]
    w = 8
    while w > 1 and ((1 << w) - 1) ** 2 * d > 2**24:
        w -= 1
    K = min(-(-bits // w), 12)
    factor = d * (3 + K * (K - 1) / 2) * 2.0 ** (-w * K)
    s = 2.0 ** (np.floor(np.log2(np.abs(A).max(axis=1))) + 1)
    mx = np.abs(X).max(axis=1)
    t = np.where(mx > 0, 2.0 ** (np.floor(np.log2(np.maximum(mx, 1e-300))) + 1), 0.0)
    return factor * t[:, None] * s[None, :]


def accumulation_bound(A, X, bits=56):
    d = A.shape[1]
    w = 8
    while w > 1 and ((1 << w) - 1) ** 2 * d > 2**24:
        w -= 1
    K = min(-(-bits // w), 12)
    N = K * (K + 1) / 2
    return N * N * 2.0**-48 * (np.abs(X) @ np.abs(A).T)


def products(A, X, NU):
    s = ess.Sampler(A, np.ones(A.shape[0]), precision=ess.ESS_PREC_FP64, **SPLIT)
    try:
        P, Q = s.products(dev(X), dev(NU))
        return host(P), host(Q)
    finally:
        s.close()


@pytest.mark.parametrize("n,m,d", [(1, 20, 10), (130, 300, 137), (64, 2001, 1000),
                                   (33, 500, 2000), (300, 130, 137), (513, 2001, 1000),
                                   (260, 200, 2000)])
def test_split_products_exact_inputs(n, m, d):
    """Entries on a 2^-12 grid below 8 in magnitude: every product and every
    sum of up to 2000 of them is exact in double, so the reference is the exact
    value; the 56-bit slices hold such entries exactly, so only the final
    rounding of the (hi, lo) float pair to double remains.  The sizes leave
    ragged chain and constraint tails; at d = 2000 the slices are 6 bits wide
    (10 per operand, 55 slice pairs)."""
    rng = np.random.default_rng(n + 5 * m + d)
    grid = lambda shape: np.round(rng.uniform(-7.9, 7.9, size=shape) * 4096) / 4096
    A, X, NU = grid((m, d)), grid((n, d)), grid((n, d))
    P, Q = products(A, X, NU)
    for V, Y in ((X, P), (NU, Q)):
        ref = V @ A.T  # exact
        err = np.abs(Y - ref)
        tol = accumulation_bound(A, V) + 2.0**-52 * np.abs(ref)
        assert np.all(err <= tol), float((err / np.maximum(tol, 1e-300)).max())


@pytest.mark.parametrize("n,m,d", [(1, 20, 10), (130, 300, 137), (300, 1000, 333),
                                   (64, 2001, 1000), (33, 500, 2000)])
def test_split_products_within_bound(n, m, d):
    """Full-precision random inputs: within the split's bound plus the final
    rounding, plus the rounding of the double reference itself (at most
    d 2^-53 sum |a||x| for a dot product of d terms)."""
    rng = np.random.default_rng(n + 3 * m + d)
    A = rng.standard_normal((m, d)) / math.sqrt(d)
    X = rng.standard_normal((n, d)) * 0.3
    NU = rng.standard_normal((n, d))
    P, Q = products(A, X, NU)
    for V, Y in ((X, P), (NU, Q)):
        ref = V @ A.T
        absdot = np.abs(V) @ np.abs(A).T
        tol = (split_bound(A, V) + accumulation_bound(A, V) + 2.0**-52 * np.abs(ref)
               + d * 2.0**-53 * absdot)
        err = np.abs(Y - ref)
        assert np.all(err <= tol), float((err / tol).max())
        # far more accurate than FP32 (a wrong slice weight would not be)
        assert np.max(err / absdot) < 1e-11


@pytest.mark.parametrize("d,m,n", [(10, 20, 16), (37, 300, 130), (100, 200, 300),
                                   (333, 1000, 257)])
def test_split_one_step_matches_oracle(d, m, n):
    rng = np.random.default_rng(d * 31 + m)
    A, b, X = feasible_instance(rng, d, m, n)
    NU = rng.standard_normal((n, d))
    U = rng.uniform(size=n)
    check_fp64(A, b, X, NU, U, **SPLIT)


@pytest.mark.parametrize("sort_threads", [0, 256])
def test_split_probit_orthant(sort_threads):
    """Equal half-widths (b = 0): every arc survives the prune."""
    rng = np.random.default_rng(4)
    k = 200
    M = rng.standard_normal((k, k))
    L = np.linalg.cholesky(M @ M.T / k + np.eye(k))
    z = rng.standard_normal(k)
    y = np.sign(L @ z)
    A = -y[:, None] * L
    check_fp64(A, np.zeros(k), np.tile(z, (32, 1)), rng.standard_normal((32, k)),
               rng.uniform(size=32), sort_threads=sort_threads, **SPLIT)


def test_split_run_reproduces_oracle_chains():
    inst = workloads.small(n_chains=16)
    Xo, _, rej_o = oracle.run(inst.A, inst.b, inst.X0, 60, seed=3)
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64, **SPLIT)
    try:
        X = dev(inst.X0)
        s.run(X, 60, seed=3)
        Xg = host(X)
        st = s.stats()
    finally:
        s.close()
    np.testing.assert_allclose(Xg, Xo, rtol=0, atol=1e-8)
    assert st["rejections"] == 0 and rej_o.sum() == 0
    assert st["max_refresh_drift"] < 1e-10


def test_split_medium_run_feasible_and_close_to_dfma():
    """A 16-step run at d = 100, m = 200: every state feasible, and the chains
    equal the DFMA form's to 1e-9 (both products FP64-class; longer runs
    drift apart chaotically from differences in the last bits)."""
    inst = workloads.medium(n_chains=256)
    out = []
    for cfg in ({}, SPLIT):
        s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64, **cfg)
        try:
            X = dev(inst.X0)
            s.run(X, 16, seed=7)
            out.append(host(X))
        finally:
            s.close()
    assert np.max(out[1] @ inst.A.T - inst.b) <= 0.0
    np.testing.assert_allclose(out[1], out[0], rtol=0, atol=1e-9)


def test_split_infeasible_start_is_refused():
    inst = workloads.small(n_chains=4)
    X0 = inst.X0.copy()
    X0[2] = 100.0
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64, **SPLIT)
    try:
        with pytest.raises(ess.EssError) as e:
            s.run(dev(X0), 5, seed=0)
        assert e.value.status == ess.ESS_ERR_INFEASIBLE_X0
    finally:
        s.close()


def test_split_start_on_the_boundary_is_accepted():
    """A start point exactly on a constraint (A x = b in FP64) is feasible; the
    split product alone cannot tell, the bounded check recomputes it."""
    rng = np.random.default_rng(9)
    d, m = 20, 40
    A = rng.standard_normal((m, d))
    x = rng.standard_normal(d) * 0.1
    b = A @ x + rng.uniform(0.1, 1.0, size=m)
    b[3] = A[3] @ x  # x lies on row 3's hyperplane (FP64 dot product)
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_FP64, **SPLIT)
    try:
        X = dev(np.tile(x, (4, 1)))
        s.run(X, 3, seed=1)
        assert np.max(host(X) @ A.T - b) <= 0.0
    finally:
        s.close()
