"""App. A's factor on the GPU (ess_cholesky) against the FP64 oracle.

The oracle's Cholesky-Banachiewicz factor is pinned in test_oracle_cholesky.
Sizes cross the 64 x 64 blocks (one block, ragged last block, many blocks);
the probit configuration's K (n = 2000, RBF + 1e-6 jitter, condition number
~4e8) is factored as the sampler's setup would.  The factor must equal the
oracle's within 1e-9 (numpy's and the oracle's differ by ~1e-11 there) and
reconstruct K; the strict upper triangle is left as it was; a matrix that is
not positive definite is refused at the right row.
"""
import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
import workloads
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 130, 517])
def test_cholesky_random_spd(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    S = M @ M.T / n + np.eye(n)
    A = dev(S)
    ess.ess_cholesky(A)
    got = host(A)
    L = np.tril(got)
    want = oracle.cholesky(S)
    np.testing.assert_allclose(L, want, rtol=0, atol=1e-12 * np.abs(want).max())
    np.testing.assert_array_equal(np.triu(got, 1), np.triu(S, 1))
    np.testing.assert_allclose(L @ L.T, S, rtol=0, atol=1e-12 * np.abs(S).max())


def test_cholesky_probit_kernel_matrix():
    K = workloads.probit(n_chains=1)["K"]
    L = host(ess.cholesky(K))
    want = oracle.cholesky(K)
    assert np.max(np.abs(L - want)) <= 1e-9
    assert np.max(np.abs(L @ L.T - K)) <= 1e-13


def test_cholesky_refuses_indefinite():
    S = np.eye(100)
    S[70, 70] = -1.0
    A = dev(S)
    with pytest.raises(ess.EssError) as e:
        ess.ess_cholesky(A)
    assert e.value.status == ess.ESS_ERR_ARG
    assert "row 70" in str(e.value)
