"""ess_hdr (normal probability P(A x <= b) by the HDR splitting estimator on
the GPU's chain steps) against the oracle's estimator with the same random
numbers.

FP64 forms: the chains follow the oracle's to rounding, so the level
decisions are the oracle's: the same number of levels, the first eight shifts
to 1e-9 relative and the same counts in those levels.  Along a level sequence
the samples descend from chains of n_between steps per level, each restarted
from a listed sample; differences in the last bits grow along that lineage
(as along any long trajectory, see test_gpu_trajectories), and once a lineage
has taken another piece its descendants are as good as independent draws: so
after ~100 steps the shifts agree to 1e-3 of the first shift, the counts and
log Z within four standard errors of the estimator.  Mixed form (float states, FP32 steps): the
estimate lies within the estimator's error of the closed form.  Closed forms:
a halfspace (Phi(b / |a|)), a box (a product of one-dimensional
probabilities), Sheppard's orthant formula 1/4 + asin(r) / (2 pi).
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


def _phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def _tol(counts, n):
    p = np.asarray(counts, dtype=float) / n
    return 4.0 * math.sqrt(3.0 * float(np.sum((1.0 - p) / (n * p))))


def _halfspace():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(4)
    return a[None, :], np.array([-3.0 * np.linalg.norm(a)]), math.log(_phi(-3.0))


def _box():
    d = 3
    A = np.vstack([np.eye(d), -np.eye(d)])
    b = np.concatenate([np.full(d, 2.5), np.full(d, -1.0)])
    return A, b, d * math.log(_phi(2.5) - _phi(1.0))


def _orthant():
    r = -0.9
    L = np.linalg.cholesky(np.array([[1.0, r], [r, 1.0]]))
    return L, np.zeros(2), math.log(0.25 + math.asin(r) / (2 * math.pi))


def _polytope():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 10))
    b = 0.8 + 0.2 * rng.standard_normal(30)
    return A, b, None


CASES = {"halfspace": _halfspace, "box": _box, "orthant": _orthant, "polytope": _polytope}
FP64_FORMS = [("dfma", {}), ("split", {"fp64_products": ess.ESS_PRODUCTS_SPLIT})]


@pytest.mark.parametrize("form,cfg", FP64_FORMS, ids=[f[0] for f in FP64_FORMS])
@pytest.mark.parametrize("case", list(CASES))
def test_hdr_fp64_equals_oracle(case, form, cfg):
    A, b, want = CASES[case]()
    n, rho, kb, seed = 1500, 0.5, 8, 17
    ref = oracle.hdr(A, b, n, rho=rho, n_between=kb, seed=seed)
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_FP64, **cfg)
    try:
        got = ess.ess_hdr(s.state, n, rho, kb, seed)
    finally:
        s.close()
    T = len(ref["shifts"])
    assert len(got["shifts"]) == T
    early = min(T, 8)
    np.testing.assert_allclose(got["shifts"][:early], ref["shifts"][:early], rtol=1e-9,
                               atol=1e-12)
    # later shifts: within 1e-3 of the first shift (the scale of the levels)
    np.testing.assert_allclose(got["shifts"], ref["shifts"], rtol=0,
                               atol=1e-3 * ref["shifts"][0] + 1e-12)
    k = math.ceil(rho * n)
    assert np.all(got["counts_ss"][:-1] == k)
    np.testing.assert_array_equal(got["counts"][:early - 1], ref["counts"][:early - 1])
    # once a lineage has diverged, its level counts are as good as independent
    # draws: within four standard errors (binomial, inflated by 3 for the
    # chains' correlation)
    p = ref["counts"] / n
    slack = 4.0 * np.sqrt(3.0 * n * p * (1.0 - p)) + 1.0
    assert np.all(np.abs(got["counts"] - ref["counts"]) <= slack)
    assert abs(got["log_z"] - ref["log_z"]) <= _tol(ref["counts"], n)
    assert abs(got["log_z_ss"] - ref["log_z_ss"]) <= _tol(ref["counts_ss"], n)
    if want is not None:
        assert abs(got["log_z"] - want) <= _tol(got["counts"], n)


@pytest.mark.parametrize("case", ["halfspace", "box", "orthant"])
def test_hdr_mixed_within_error(case):
    A, b, want = CASES[case]()
    n = 4096
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_MIXED)
    try:
        got = ess.ess_hdr(s.state, n, 0.5, 8, 29)
    finally:
        s.close()
    assert got["shifts"][-1] == 0.0 and np.all(np.diff(got["shifts"]) < 0)
    assert abs(got["log_z"] - want) <= _tol(got["counts"], n), (got["log_z"], want)
    assert abs(got["log_z_ss"] - want) <= _tol(got["counts_ss"], n)


def test_hdr_single_level_and_state_reuse():
    """Z above rho: one level, plain Monte Carlo over the stage-2 draws, the
    oracle's count; afterwards the state's b is the original one again (a
    step through ess_run matches the oracle's run)."""
    A = np.array([[1.0, 0.5], [-0.3, 1.0]])
    b = np.array([1.2, 1.5])
    n = 1000
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_FP64)
    try:
        got = ess.ess_hdr(s.state, n, 0.4, 4, 3)
        X0 = np.zeros((8, 2))
        X = dev(X0)
        s.run(X, 5, seed=9)
        Xg = host(X)
    finally:
        s.close()
    ref = oracle.hdr(A, b, n, rho=0.4, n_between=4, seed=3)
    assert list(got["shifts"]) == [0.0] == list(ref["shifts"])
    assert got["counts"][0] == ref["counts"][0]
    np.testing.assert_allclose(Xg, oracle.run(A, b, X0, 5, seed=9)[0], rtol=0, atol=1e-12)


def test_hdr_errors():
    A = np.array([[1.0], [-1.0]])
    s = ess.Sampler(A, np.array([-1.0, -1.0]), precision=ess.ESS_PREC_FP64)  # empty: x <= -1, x >= 1
    try:
        with pytest.raises(ess.EssError) as e:
            ess.ess_hdr(s.state, 200, 0.5, 2, 1, max_levels=6)
        assert e.value.status == ess.ESS_ERR_UNSUPPORTED
        for bad in (dict(n_samples=1), dict(rho=0.0), dict(rho=1.0), dict(n_between=0),
                    dict(rho=0.999)):
            kw = dict(n_samples=200, rho=0.5, n_between=2)
            kw.update(bad)
            with pytest.raises(ess.EssError) as e:
                ess.ess_hdr(s.state, kw["n_samples"], kw["rho"], kw["n_between"], 1)
            assert e.value.status == ess.ESS_ERR_ARG
    finally:
        s.close()
