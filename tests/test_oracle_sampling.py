"""Pins of the oracle's random draws, theta draw and chain (Alg. 1).

* The theta draw is the inverse CDF of the uniform law on I_act: checked by
  the measure identity |I_act and [0, theta(u)]| = u |I_act| and monotonicity.
* Box-Muller normals and the uniforms are checked against their laws (KS).
* The Philox bit stream is pinned in test_oracle_philox.py, against an
  independent library implementation.  The second implementation written
  here restates the same round function from the same source, so agreeing
  with it only cross-checks the C transcription (word order, carries); the
  uniformity and normality tests below check the generator's laws.
* The chain's stationary law is the truncated normal (Sec. 2, citing Murray
  et al.): KS tests against the exact univariate truncated normal at d = 1 and
  d = 2, and the moments printed in the Sec. 4.1 table.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads
from conftest import read_golden

PI = math.pi


def test_theta_inverse_cdf_measure_identity():
    rng = np.random.default_rng(11)
    for _ in range(200):
        k = int(rng.integers(1, 6))
        cuts = np.sort(rng.uniform(0, 2 * PI, size=2 * k))
        pieces = cuts.reshape(k, 2)
        lens = pieces[:, 1] - pieces[:, 0]
        total = lens.sum()
        prev = -1.0
        for u in np.linspace(0.0, 0.999999, 37):
            th = oracle.draw_theta(pieces, u)
            assert any(lo <= th <= hi for lo, hi in pieces)
            below = sum(max(0.0, min(hi, th) - lo) for lo, hi in pieces)
            assert below == pytest.approx(u * total, abs=1e-12)
            assert th >= prev
            prev = th


def test_theta_empty_set_stays():
    assert oracle.draw_theta(np.array([[0.0, 0.0], [2 * PI, 2 * PI]]), 0.4) == 0.0


def _py_philox(ctr, key):
    """Second transcription of the Philox4x32-10 round function (Salmon et al.
    2011): a cross-check of the C code, not a pin of the constants."""
    mask = 0xFFFFFFFF
    c = [int(v) for v in ctr]
    k = [int(v) for v in key]
    for _ in range(10):
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & mask, p1 & mask,
             ((p0 >> 32) ^ c[3] ^ k[1]) & mask, p0 & mask]
        k = [(k[0] + 0x9E3779B9) & mask, (k[1] + 0xBB67AE85) & mask]
    return c


def test_philox_cross_implementation():
    rng = np.random.default_rng(3)
    for _ in range(500):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64)
        got = oracle.philox4x32_10(ctr.astype(np.uint32), key.astype(np.uint32))
        assert [int(v) for v in got] == _py_philox(ctr, key)


def test_philox_counter_layout():
    seed = 0x123456789ABCDEF0
    blk = oracle.rng_block(seed, 5, 7, 11, problem=3, stream=1)
    ref = _py_philox([5, 7, 11, (3 << 8) | 1], [seed & 0xFFFFFFFF, seed >> 32])
    assert [int(v) for v in blk] == ref


def test_uniform_bits_law():
    words = np.array([oracle.rng_block(0, n, 0, 0) for n in range(20000)], dtype=np.uint64)
    u = (words.ravel().astype(np.float64) + 0.5) / 2**32
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # each bit is fair
    bits = ((words.ravel()[:, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.01)


def test_box_muller_normals():
    z = np.concatenate([oracle.draw_nu(42, c, t, 101) for c in range(40) for t in range(10)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 6 * math.sqrt(2 / z.size)
    # partial block: the first d entries do not depend on d
    assert np.array_equal(oracle.draw_nu(1, 2, 3, 7), oracle.draw_nu(1, 2, 3, 9)[:7])


def test_theta_uniforms():
    u = np.array([oracle.draw_u(9, c, t) for c in range(200) for t in range(50)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3


# --------------------------------------------------------------------------
# Stationary law: exact truncated normal
# --------------------------------------------------------------------------

def _final_states(inst, n_iter, seed=0):
    X, _, rej = oracle.run(inst.A, inst.b, inst.X0, n_iter, seed)
    return X, rej


def test_chain_d1_interval_ks():
    inst = workloads.interval(-0.5, 1.2, n_chains=8192)
    X, rej = _final_states(inst, 60)
    law = stats.truncnorm(-0.5, 1.2)
    assert stats.kstest(X[:, 0], law.cdf).pvalue > 1e-3
    assert X[:, 0].mean() == pytest.approx(0.273909, abs=5 * math.sqrt(0.215291 / 8192))
    assert law.mean() == pytest.approx(0.273909, abs=1e-6)
    assert rej.sum() == 0


def test_chain_d2_box_ks():
    inst = workloads.box2(n_chains=8192)
    X, rej = _final_states(inst, 200, seed=5)
    assert stats.kstest(X[:, 0], stats.truncnorm(-1.0, 3.0).cdf).pvalue > 1e-3
    assert stats.kstest(X[:, 1], stats.truncnorm(-0.5, 1.2).cdf).pvalue > 1e-3
    assert abs(np.corrcoef(X[:, 0], X[:, 1])[0, 1]) < 5 / math.sqrt(8192)
    assert rej.sum() == 0


@pytest.mark.parametrize("row", read_golden("table_univariate.txt"), ids=lambda r: f"{r[1]}_{r[2]}")
def test_chain_matches_paper_table(row):
    lo, hi, mu, var = (float(v) for v in row[1:])
    # printed values agree with the closed form to the printed digits
    law = stats.truncnorm(lo, hi)
    assert law.mean() == pytest.approx(mu, abs=5e-5)
    assert law.var() == pytest.approx(var, abs=5e-5)
    inst = workloads.interval(lo, hi, n_chains=4096, x0=0.5 * (lo + hi))
    X, samples, rej = oracle.run(inst.A, inst.b, inst.X0, 300, seed=2, record_every=10)
    kept = samples[:, 10:, 0].ravel()   # 100 burn-in iterations dropped
    n_eff = 4096 * 5  # conservative effective sample count
    assert kept.mean() == pytest.approx(mu, abs=5 * math.sqrt(var / n_eff) + 5e-5)
    assert kept.var() == pytest.approx(var, rel=0.05, abs=5e-5)
    assert np.all(kept >= lo) and np.all(kept <= hi)
    assert rej.sum() == 0   # FP64: the paper reports no violation in double precision


def test_every_iterate_feasible_small():
    inst = workloads.small(n_chains=16, n_iter=200)
    X, samples, rej = oracle.run(inst.A, inst.b, inst.X0, 200, seed=0, record_every=1)
    S = samples.reshape(-1, inst.d)
    assert np.max(S @ inst.A.T - inst.b) <= 0.0
    assert rej.sum() == 0


def test_run_is_resumable():
    inst = workloads.small(n_chains=4)
    X_full, _, _ = oracle.run(inst.A, inst.b, inst.X0, 30, seed=9)
    X_half, _, _ = oracle.run(inst.A, inst.b, inst.X0, 12, seed=9)
    X_rest, _, _ = oracle.run(inst.A, inst.b, X_half, 18, seed=9, t0=12)
    assert np.array_equal(X_full, X_rest)


# --------------------------------------------------------------------------
# App. A: whitening
# --------------------------------------------------------------------------

def test_whiten_identity():
    rng = np.random.default_rng(4)
    d, m = 5, 9
    A = rng.standard_normal((m, d))
    b = rng.uniform(0.5, 1.0, size=m)
    mu = rng.standard_normal(d)
    M = rng.standard_normal((d, d))
    L = np.linalg.cholesky(M @ M.T + d * np.eye(d))
    Aw, bw = oracle.whiten(A, b, mu, L)
    U = rng.standard_normal((50, d))
    Xu = oracle.unwhiten(L, mu, U)
    np.testing.assert_allclose(Xu, U @ L.T + mu, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(U @ Aw.T - bw, Xu @ A.T - b, rtol=1e-12, atol=1e-12)


def test_whiten_diagonal_closed_form():
    # N(mu, diag(s^2)) truncated to a box: marginals are scaled truncated normals
    mu = np.array([0.5, -1.0])
    s = np.array([2.0, 0.5])
    A0 = np.vstack([np.eye(2), -np.eye(2)])
    lo = np.array([-1.0, -1.2])
    hi = np.array([2.0, -0.7])
    b0 = np.concatenate([hi, -lo])
    Aw, bw = oracle.whiten(A0, b0, mu, np.diag(s))
    U0 = np.tile((0.5 * (lo + hi) - mu) / s, (8192, 1))
    U, _, _ = oracle.run(Aw, bw, U0, 60, seed=13)
    X = oracle.unwhiten(np.diag(s), mu, U)
    for j in range(2):
        law = stats.truncnorm((lo[j] - mu[j]) / s[j], (hi[j] - mu[j]) / s[j], loc=mu[j], scale=s[j])
        assert stats.kstest(X[:, j], law.cdf).pvalue > 1e-3


def test_rejection_safeguard_at_piece_endpoints():
    """Sec. 3.3: an infeasible x_{t+1} is rejected and the chain stays at x_t.

    Draws u so that theta lands on a piece endpoint, where a_i.x(theta) = b_i
    holds exactly in real arithmetic and rounding decides the residual's sign.
    Every emitted iterate must be feasible; every rejection must return x_t;
    and the rounding must trigger the safeguard at least once."""
    rng = np.random.default_rng(21)
    n_rej = 0
    for _ in range(400):
        d = int(rng.integers(2, 6))
        m = int(rng.integers(2, 12))
        A = rng.standard_normal((m, d))
        x = rng.standard_normal(d)
        b = A @ x + rng.uniform(0.0, 0.5, size=m)
        nu = rng.standard_normal(d) * 2.0
        pcs = oracle.step(A, b, x, nu, 0.0).pieces
        lens = pcs[:, 1] - pcs[:, 0]
        total = lens.sum()
        cum = np.concatenate([[0.0], np.cumsum(lens)])
        for j in range(1, pcs.shape[0]):
            for k in range(-2, 3):
                u = min(max(cum[j] / total + k * 2.0**-52, 0.0), 1.0 - 2.0**-53)
                res = oracle.step(A, b, x, nu, u)
                if res.rejected:
                    n_rej += 1
                    assert np.array_equal(res.x_next, x)
                else:
                    assert oracle.max_residual(A, b, res.x_next) <= 0.0
    assert n_rej > 0
