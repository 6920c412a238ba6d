"""The streamed chain-step kernel (one warp per chain, p and q rows streamed
through shared memory in chunks by bulk copies) against the FP64 oracle and
the warp kernel that reads the rows from global memory.

Mixed form, grid inputs (exact P and Q, see gpu_helpers.grid_instance), the
a-priori exemption of test_gpu_mixed_step.check_mixed: pieces endpoint by
endpoint, theta and x' within 1e-5 rad.  Shapes cover m below the first-batch
size (no first batch), m = 4096 (the largest staged row), d = 4, chain counts
below and above the persistent grid with a ragged tail, m not a multiple of
the chunk, and chains whose arcs all survive the prune (every chain handed to
the CTA-per-chain kernel).  Runs through the streamed kernel and through the
warp kernel agree to the FP32 rounding of the step.
"""
import math

import numpy as np
import pytest

import paper_2407_10449_gb300 as ess
import workloads
from gpu_helpers import dev, host, grid_instance, grid_bits, to_grid
from test_gpu_mixed_step import check_mixed

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,m,n", [(4, 8, 5), (12, 100, 300), (64, 252, 1000), (100, 200, 256),
                                   (128, 1024, 700), (16, 4096, 40), (1000, 2000, 97),
                                   (40, 516, 333), (8, 260, 64)])
def test_stream_step_parity(d, m, n):
    rng = np.random.default_rng(7 * d + m)
    A, b, X, NU = grid_instance(rng, d, m, n, scale=1.0 / math.sqrt(d), slack=(0.05, 0.6))
    U = rng.uniform(size=n)
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_MIXED)
    try:
        ess.ess_set_chain_kernel(s.state, ess.ESS_CHAIN_STREAM)
        assert ess.ess_get_chain_kernel(s.state) == ess.ESS_CHAIN_STREAM
    finally:
        s.close()
    check_mixed(A, b, X, NU, U, chain_kernel=ess.ESS_CHAIN_STREAM)


def test_stream_overflow_to_cta_kernel():
    """A probit-style orthant (b = 0: every arc has half-width pi / 2, none
    contains another): every chain has more survivors than a warp sorts and
    goes to the CTA-per-chain kernel."""
    rng = np.random.default_rng(9)
    k = 160
    M = rng.standard_normal((k, k))
    B = grid_bits(k)
    L = to_grid(np.linalg.cholesky(M @ M.T / k + np.eye(k)), B)
    z = to_grid(rng.standard_normal(k), B)
    f = L @ z
    assert np.all(f != 0.0)
    A = -np.sign(f)[:, None] * L
    n = 48
    X = np.tile(z, (n, 1))
    NU = to_grid(rng.standard_normal((n, k)), B)
    U = rng.uniform(size=n)
    check_mixed(A, np.zeros(k), X, NU, U, chain_kernel=ess.ESS_CHAIN_STREAM)


def _run(inst, kind, n_iter, seed, graphs=True):
    import torch
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_MIXED, refresh_k=8)
    try:
        ess.ess_set_chain_kernel(s.state, kind)
        ess.ess_set_graphs(s.state, graphs)
        X = dev(inst.X0)
        s.run(X, n_iter, seed=seed)
        k = ess.ess_get_chain_kernel(s.state)
        st = s.stats()
        return host(X), k, st
    finally:
        s.close()


def test_stream_and_warp_kernels_agree_on_a_run():
    """Medium workload, 20 steps: the two kernels' chains agree to the FP32
    rounding of the step (the same map, FP32 operations in another order);
    graph replay and plain launches of the streamed kernel are bit-identical."""
    inst = workloads.medium(n_chains=512)
    Xc, kc, stc = _run(inst, ess.ESS_CHAIN_STREAM, 20, 3)
    Xw, kw, stw = _run(inst, ess.ESS_CHAIN_WARP, 20, 3)
    Xp, _, _ = _run(inst, ess.ESS_CHAIN_STREAM, 20, 3, graphs=False)
    assert kc == ess.ESS_CHAIN_STREAM and kw == ess.ESS_CHAIN_WARP
    np.testing.assert_array_equal(Xc, Xp)
    gap = np.max(np.abs(Xc - Xw) / (1.0 + np.abs(Xw)), axis=1)
    assert np.median(gap) < 1e-5 and np.mean(gap < 1e-4) > 0.95, (np.median(gap), gap.max())
    assert np.max(Xc @ inst.A.T - inst.b) <= 0.0
    assert stc["numeric_errors"] == 0 and stc["sort_keys"] > 0


def test_stream_records_samples():
    """Recorded samples through the streamed kernel equal the states."""
    import torch
    inst = workloads.medium(n_chains=64)
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_MIXED)
    try:
        ess.ess_set_chain_kernel(s.state, ess.ESS_CHAIN_STREAM)
        X = dev(inst.X0)
        S = torch.zeros((64, 3, inst.d), dtype=torch.float32, device="cuda")
        s.run(X, 6, seed=2, samples=S, record_every=2)
        np.testing.assert_array_equal(host(S[:, 2]).astype(np.float64), host(X))
        assert np.max(host(S).reshape(-1, inst.d) @ inst.A.T - inst.b) <= 0.0
    finally:
        s.close()


def test_chain_kernel_setter_rejects_unknown_kinds():
    s = ess.Sampler(np.eye(4), np.ones(4), precision=ess.ESS_PREC_MIXED)
    try:
        for bad in (-1, 3, 7):
            with pytest.raises(ess.EssError):
                ess.ess_set_chain_kernel(s.state, bad)
    finally:
        s.close()
