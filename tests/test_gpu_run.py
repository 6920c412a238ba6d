"""Chains run on the GPU (ess_run): draws, reproducibility and the stationary law.

* Philox blocks are bit-identical to the oracle's independent implementation;
  the normals agree to the precision of each form.
* FP64 runs reproduce the oracle's chains (same seed, same counters).
* Every emitted iterate is feasible in FP64 (Sec. 3.3), for both forms.
* The stationary law is the truncated normal (KS at d = 1 and d = 2; the
  Sec. 4.1 table's moments).
* A run split at a multiple of refresh_k reproduces the unsplit run.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import paper_2407_10449_gb300 as ess
import workloads
from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu

FORMS = [ess.ESS_PREC_FP64, ess.ESS_PREC_MIXED]


def test_philox_bit_exact():
    import torch
    for seed, chain, t, prob, stream in [(0, 0, 0, 0, 0), (1, 5, 7, 0, 1), (2**63 + 11, 123456, 99, 3, 0),
                                         (0xDEADBEEFCAFE, 2**32 - 1, 2**31, 0xFFFFFF, 255)]:
        out = torch.zeros((300, 4), dtype=torch.int32, device="cuda")
        ess.ess_philox_blocks(seed, chain, t, prob, stream, 300, out)
        got = host(out).view(np.uint32)
        want = np.array([oracle.rng_block(seed, n, chain, t, prob, stream) for n in range(300)])
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("form", FORMS)
def test_normals_match_oracle(form):
    A = np.eye(37)
    s = ess.Sampler(A, np.ones(37), precision=form)
    try:
        z = host(s.draw_normals(50, 11, 777)).astype(np.float64)
    finally:
        s.close()
    want = np.stack([oracle.draw_nu(777, c, 11, 37) for c in range(50)])
    tol = 1e-13 if form == ess.ESS_PREC_FP64 else 2e-6
    assert np.all(np.abs(z - want) <= tol * (1 + np.abs(want)))


def test_fp64_run_reproduces_oracle_chains():
    inst = workloads.small(n_chains=16)
    Xo, _, rej_o = oracle.run(inst.A, inst.b, inst.X0, 60, seed=3)
    s = ess.Sampler(inst.A, inst.b, precision=ess.ESS_PREC_FP64)
    try:
        X = dev(inst.X0)
        s.run(X, 60, seed=3)
        Xg = host(X)
        st = s.stats()
    finally:
        s.close()
    np.testing.assert_allclose(Xg, Xo, rtol=0, atol=1e-8)
    assert st["rejections"] == 0 and rej_o.sum() == 0


@pytest.mark.parametrize("form", FORMS)
def test_split_run_is_bit_identical(form):
    inst = workloads.medium(n_chains=64)
    s = ess.Sampler(inst.A, inst.b, precision=form, refresh_k=8)
    try:
        Xa = dev(inst.X0)
        s.run(Xa, 48, seed=5)
        Xb = dev(inst.X0)
        s.run(Xb, 16, seed=5)
        s.run(Xb, 32, seed=5, t0=16)
        np.testing.assert_array_equal(host(Xa), host(Xb))
    finally:
        s.close()


@pytest.mark.parametrize("form", FORMS)
def test_graph_replay_is_bit_identical(form):
    """Refresh periods replayed from a CUDA graph give the chains of plain
    launches, bit for bit (start off a period boundary, end inside one)."""
    inst = workloads.medium(n_chains=96)
    out = []
    for graphs in (True, False):
        s = ess.Sampler(inst.A, inst.b, precision=form, refresh_k=8)
        try:
            ess.ess_set_graphs(s.state, graphs)
            X = dev(inst.X0)
            s.run(X, 45, seed=7, t0=3)
            out.append(host(X))
            n_graph = ess.ess_graph_launches(s.state)
        finally:
            s.close()
        # steps 3..47: steps 3..7 run plain, the periods starting at 8, 16, 24,
        # 32 and 40 replay
        assert n_graph == (5 if graphs else 0)
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("form", FORMS)
def test_draws_ahead_are_bit_identical(form):
    """nu of step t + 1 drawn on a side stream beside step t (plain launches
    and replayed periods) gives the chains of strictly sequential launches
    (per-phase timing on: every draw in line), bit for bit."""
    inst = workloads.medium(n_chains=80)
    out = []
    for timing, graphs in ((True, False), (False, False), (False, True)):
        s = ess.Sampler(inst.A, inst.b, precision=form, refresh_k=8)
        try:
            ess.ess_set_graphs(s.state, graphs)
            ess.ess_set_timing(s.state, timing)
            X = dev(inst.X0)
            s.run(X, 37, seed=11, t0=5)
            out.append(host(X))
        finally:
            s.close()
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[0], out[2])


@pytest.mark.parametrize("form", FORMS)
def test_steps_capture_into_a_cuda_graph(form):
    """ess_chains_step enqueued while the caller captures its stream (the
    internal work and draw streams fork from it and join back): one replay of
    the captured steps, across a refresh boundary, gives the chains of the
    same steps launched directly."""
    import torch
    inst = workloads.medium(n_chains=64)
    out = []
    for capture in (False, True):
        s = ess.Sampler(inst.A, inst.b, precision=form, refresh_k=8)
        try:
            ess.ess_set_graphs(s.state, False)
            st = torch.cuda.Stream()
            X = dev(inst.X0)
            ess.ess_chains_init(s.state, X, 64, 3, stream=st)
            ess.ess_chains_step(s.state, 2, 9, stream=st)  # steps 3, 4
            if capture:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=st):
                    ess.ess_chains_step(s.state, 4, 9, stream=st)  # steps 5 .. 8
                g.replay()
            else:
                ess.ess_chains_step(s.state, 4, 9, stream=st)
            torch.cuda.synchronize()
            ess.ess_chains_get(s.state, X, stream=st)
            out.append(host(X))
        finally:
            s.close()
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("form", FORMS)
def test_autotune_keeps_the_chains(form):
    """The autotuner times its candidates without moving any chain: a tuned
    run equals an untuned run with the same sort path (the q GEMM's tile
    width does not change any element's sums)."""
    inst = workloads.medium(n_chains=200)
    s = ess.Sampler(inst.A, inst.b, precision=form, autotune=1)
    try:
        Xa = dev(inst.X0)
        s.run(Xa, 12, seed=4)
        width, sort_threads = ess.ess_get_tuning(s.state)
        st = s.stats()
    finally:
        s.close()
    if form == ess.ESS_PREC_MIXED:
        assert width in (64, 128, 160, 192, 224, 256, 2128, 2160, 2192, 2224, 2256,
                         3128, 3160, 3192, 3224, 3256)
    else:
        assert width == 0
    assert sort_threads in (0, 32, 64, 128)
    assert st["steps"] == 200 * 12
    s = ess.Sampler(inst.A, inst.b, precision=form, sort_threads=sort_threads)
    try:
        Xb = dev(inst.X0)
        s.run(Xb, 12, seed=4)
    finally:
        s.close()
    np.testing.assert_array_equal(host(Xa), host(Xb))


@pytest.mark.parametrize("form", FORMS)
def test_every_iterate_feasible(form):
    inst = workloads.medium(n_chains=128)
    import torch
    s = ess.Sampler(inst.A, inst.b, precision=form)
    try:
        X = dev(inst.X0)
        S = torch.zeros((128, 150, inst.d), dtype=s.sample_dtype, device="cuda")
        s.run(X, 150, seed=1, samples=S, record_every=1)
        S = host(S).astype(np.float64).reshape(-1, inst.d)
        st = s.stats()
    finally:
        s.close()
    assert np.max(S @ inst.A.T - inst.b) <= 0.0
    assert st["numeric_errors"] == 0
    assert st["steps"] == 128 * 150


@pytest.mark.parametrize("form", FORMS)
def test_ks_interval_d1(form):
    inst = workloads.interval(-0.5, 1.2, n_chains=16384)
    s = ess.Sampler(inst.A, inst.b, precision=form)
    try:
        X = dev(inst.X0)
        s.run(X, 60, seed=11)
        x = host(X)[:, 0]
    finally:
        s.close()
    assert stats.kstest(x, stats.truncnorm(-0.5, 1.2).cdf).pvalue > 1e-3


@pytest.mark.parametrize("form", FORMS)
def test_ks_box_d2(form):
    inst = workloads.box2(n_chains=16384)
    s = ess.Sampler(inst.A, inst.b, precision=form)
    try:
        X = dev(inst.X0)
        s.run(X, 200, seed=12)
        x = host(X)
    finally:
        s.close()
    assert stats.kstest(x[:, 0], stats.truncnorm(-1.0, 3.0).cdf).pvalue > 1e-3
    assert stats.kstest(x[:, 1], stats.truncnorm(-0.5, 1.2).cdf).pvalue > 1e-3
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 5 / math.sqrt(16384)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("lo,hi,mu,var", [(-1.0, 3.0, 0.2828, 0.6161), (15.0, 16.0, 15.0661, 0.0043)])
def test_paper_table_moments(form, lo, hi, mu, var):
    """Sec. 4.1: 2000 chains, 500 burn-in, thinning 10 (here 100 thinned draws each)."""
    import torch
    inst = workloads.interval(lo, hi, n_chains=2000, x0=0.5 * (lo + hi))
    s = ess.Sampler(inst.A, inst.b, precision=form)
    try:
        X = dev(inst.X0)
        s.run(X, 500, seed=21)
        S = torch.zeros((2000, 100, 1), dtype=s.sample_dtype, device="cuda")
        s.run(X, 1000, seed=21, t0=500, samples=S, record_every=10)
        x = host(S).astype(np.float64).ravel()
        st = s.stats()
    finally:
        s.close()
    assert np.all(x >= lo) and np.all(x <= hi)
    assert x.mean() == pytest.approx(mu, abs=5 * math.sqrt(var / 20000) + 5e-5)
    assert x.var() == pytest.approx(var, rel=0.05, abs=5e-5)
    if form == ess.ESS_PREC_FP64:
        assert st["rejections"] == 0


def test_infeasible_start_is_refused():
    inst = workloads.small(n_chains=4)
    X0 = inst.X0.copy()
    X0[2] = 100.0
    s = ess.Sampler(inst.A, inst.b)
    try:
        with pytest.raises(ess.EssError) as e:
            s.run(dev(X0), 5, seed=0)
        assert e.value.status == ess.ESS_ERR_INFEASIBLE_X0
    finally:
        s.close()


def test_run_host_matches_device_run():
    inst = workloads.small(n_chains=8)
    s = ess.Sampler(inst.A, inst.b)
    try:
        Xd = dev(inst.X0)
        s.run(Xd, 20, seed=4)
        Xh = np.array(inst.X0, dtype=np.float64, order="C")
        ess.ess_run_host(s.state, Xh, 8, 0, 20, 4)
        np.testing.assert_array_equal(host(Xd), Xh)
    finally:
        s.close()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n_iter,record_every", [(70, 10), (40, 7), (33, 40), (64, 32)])
def test_run_host_records_like_device_run(form, n_iter, record_every):
    """ess_run_host (host buffers; each record copied to the host from a device
    slot while the next steps run) gives the same final states and the same
    recorded samples, bit for bit, as ess_run on device buffers (samples
    written by the step kernel), for record intervals that do and do not
    divide refresh_k = 32."""
    import torch
    inst = workloads.medium(n_chains=300)
    n, d = 300, inst.d
    n_rec = n_iter // record_every
    dt = torch.float64 if form == ess.ESS_PREC_FP64 else torch.float32
    s = ess.Sampler(inst.A, inst.b, precision=form)
    try:
        Xd = dev(inst.X0)
        Sd = torch.zeros((n, max(n_rec, 1), d), dtype=dt, device="cuda")
        ess.ess_run(s.state, Xd, n, 3, n_iter, 9, Sd if n_rec else None, record_every if n_rec else 0)
        Xh = np.array(inst.X0, dtype=np.float64, order="C")
        Sh = torch.zeros((n, max(n_rec, 1), d), dtype=dt).pin_memory()
        ess.ess_run_host(s.state, Xh, n, 3, n_iter, 9, Sh.numpy() if n_rec else None,
                         record_every if n_rec else 0)
    finally:
        s.close()
    np.testing.assert_array_equal(host(Xd), Xh)
    if n_rec:
        np.testing.assert_array_equal(host(Sd), Sh.numpy())
