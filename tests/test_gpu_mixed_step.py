"""Mixed form: the FP16x3 tensor-core GEMM and the FP32 step vs the FP64 oracle.

Bar (stated for the mixed form): interval endpoints and theta within 1e-5 rad
and zero infeasible iterates.  The one-step comparisons run on grid inputs
(gpu_helpers.grid_instance) on which P = A x and Q = A nu are exact in the
mixed form, so the only differences from the FP64 oracle come from the FP32
root arithmetic.  A chain is exempted only by an a-priori bound computed from
the inputs (gpu_helpers.mixed_endpoint_bounds, App. B: h = arccos(b / r) is
ill-conditioned as |b / r| -> 1, and the kernel takes b / r in FP32 for
|b / r| <= 1 - 1e-4): if an arc endpoint that can reach an endpoint of the
active pieces has a conditioning bound above 5e-6 rad.  Every other chain
must match the oracle's pieces endpoint by endpoint, theta and x' within the
bar.  The accuracy of the products themselves on arbitrary float inputs is
checked separately against their proven bounds.  Inputs are rounded to float
first on both sides, exactly as the mixed form stores them.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess
from conftest import read_golden
from gpu_helpers import dev, host, oracle_steps, positive_pieces, fp16x3_bound, \
    sym_diff_measure, f32, grid_bits, to_grid, grid_instance, mixed_endpoint_bounds, mixed_exempt

pytestmark = pytest.mark.gpu

ANG_TOL = 1e-5


def q_error_bound(A, NU):
    """The FP16x3 GEMM's bound (see gpu_helpers.fp16x3_bound)."""
    return fp16x3_bound(A, NU)


@pytest.mark.parametrize("n,m,d", [(1, 20, 10), (130, 300, 137), (256, 448, 64),
                                   (200, 1000, 333), (128, 2000, 1000), (77, 4100, 50),
                                   (300, 130, 137), (513, 2001, 1000)])
def test_products_tensor_core_gemm(n, m, d):
    """q = A nu from the tcgen05 FP16x3 GEMM vs FP64, and p = A x (refresh) vs FP64."""
    rng = np.random.default_rng(n * 7 + m)
    A = rng.standard_normal((m, d)) / math.sqrt(d)
    b = np.ones(m)
    X = f32(rng.standard_normal((n, d)) * 0.01)
    NU = f32(rng.standard_normal((n, d)))
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_MIXED)
    try:
        P, Q = s.products(dev(X), dev(NU))
        P, Q = host(P), host(Q)
    finally:
        s.close()
    A32 = f32(A)
    q_ref = NU.astype(np.float64) @ A32.astype(np.float64).T
    err = np.abs(Q - q_ref)
    bound = q_error_bound(A32, NU)
    assert np.all(err <= bound), float((err / bound).max())
    # typical error far below the bound (a wrong operand layout would not be)
    assert np.median(err / np.maximum(bound, 1e-300)) < 0.2
    # p = A x by the exact-split refresh: within its stated bound (truncated
    # fixed-point slices) plus one rounding to float
    p_ref = X @ A.T
    tol = np.abs(p_ref) * 2.0**-23 + refresh_bound(A, X)
    assert np.all(np.abs(P - p_ref) <= tol), float(np.max(np.abs(P - p_ref) / tol))


Q_TILES = [64, 128, 160, 192, 224, 256, 2128, 2160, 2192, 2224, 2256,
           3128, 3160, 3192, 3224, 3256]


@pytest.mark.parametrize("q_tile", Q_TILES)
@pytest.mark.parametrize("n,m,d", [(513, 1000, 333), (256, 448, 64), (40, 300, 1000),
                                   (1300, 1001, 77)])
def test_q_gemm_every_tile(q_tile, n, m, d):
    """Every tile form of the q GEMM (one SM per 128-chain tile; an SM pair per
    256-chain tile with tcgen05 cta_group::2, one launch per tile or the
    persistent kernel with TMA-stored Q) within the FP16x3 bound, on ragged
    chain counts (a cluster row with one live chain), ragged m and K; m = 1001
    (rows of Q not a multiple of 16 bytes) takes the per-tile launch."""
    rng = np.random.default_rng(n + m + q_tile)
    A = rng.standard_normal((m, d)) / math.sqrt(d)
    NU = f32(rng.standard_normal((n, d)))
    X = np.zeros((n, d))
    s = ess.Sampler(A, np.ones(m), precision=ess.ESS_PREC_MIXED, q_tile=q_tile)
    try:
        _, Q = s.products(dev(X), dev(NU))
        Q = host(Q)
    finally:
        s.close()
    A32 = f32(A)
    q_ref = NU @ A32.T
    err = np.abs(Q - q_ref)
    bound = q_error_bound(A32, NU)
    assert np.all(err <= bound), float((err / bound).max())
    assert np.median(err / np.maximum(bound, 1e-300)) < 0.2


def test_q_tile_rejects_unknown_codes():
    for bad in (1, 96, 2064, 2000, 3000, 3064, 4224, -1):
        with pytest.raises(ess.EssError):
            ess.Sampler(np.eye(3), np.ones(3), precision=ess.ESS_PREC_MIXED, q_tile=bad)


def refresh_bound(A, X):
    """|p_refresh - A x| bound of the exact-split refresh: w-bit slices with
    (2^w - 1)^2 d <= 2^24, K = ceil(35 / w) slices per operand, per-row and
    per-chain power-of-two scales s_i > max |a_i|, t_c > max |x_c|."""
    d = A.shape[1]
    w = 8
    while w > 1 and ((1 << w) - 1) ** 2 * d > 2**24:
        w -= 1
    K = min(-(-35 // w), 7)
    factor = d * (3 + K * (K - 1) / 2) * 2.0 ** (-w * K)
    s = 2.0 ** (np.floor(np.log2(np.abs(A).max(axis=1))) + 1)
    mx = np.abs(X.astype(np.float32)).max(axis=1).astype(np.float64)
    t = np.where(mx > 0, 2.0 ** (np.floor(np.log2(np.maximum(mx, 1e-300))) + 1), 0.0)
    return factor * t[:, None] * s[None, :]


LIMIT = 0.5 * ANG_TOL


def check_mixed(A, b, X, NU, U, trim_eps=0.0, eps_p=0.0, eps_q=0.0, sample=None,
                max_pieces=None, max_exempt_frac=0.05, chain_kernel=None, **cfg):
    """One mixed step with given draws vs the oracle's one-step map.

    Exemptions are chosen before the GPU runs, from the inputs alone
    (mixed_endpoint_bounds, with eps_p / eps_q the a-priori product error
    bounds: zero on grid inputs).  Returns (stats, exempt count, compared)."""
    X, NU = f32(X), f32(NU)
    n = X.shape[0]
    idx = np.arange(n) if sample is None else np.asarray(sample)
    refs = oracle_steps(A, b, X[idx], NU[idx], U[idx], trim_eps)
    amp, arith = mixed_endpoint_bounds(A, b, X[idx], NU[idx], eps_p, eps_q)
    exempt = mixed_exempt(refs, amp, arith, LIMIT, trim_eps)
    s = ess.Sampler(A, b, precision=ess.ESS_PREC_MIXED, trim_eps=trim_eps, **cfg)
    try:
        if chain_kernel is None and not cfg.get("sort_threads"):
            # the warp-per-chain kernel (the default picks a CTA per chain for
            # fewer chains than SMs)
            chain_kernel = ess.ESS_CHAIN_WARP
        if chain_kernel is not None:
            ess.ess_set_chain_kernel(s.state, chain_kernel)
        mp = max_pieces or (A.shape[0] + 2)
        Xn, th, pcs, npc, rej = s.step_with_draws(dev(X), dev(NU), dev(U), max_pieces=mp)
        Xn, th, pcs, npc, rej = host(Xn), host(th), host(pcs), host(npc), host(rej)
        stats = s.stats()
    finally:
        s.close()
    # zero infeasible iterates, decided in FP64 on the float states
    assert np.max(Xn @ A.T - b[None, :]) <= 0.0
    for k, (c, r) in enumerate(zip(idx, refs)):
        if exempt[k]:
            continue
        assert npc[c] <= pcs.shape[1], c
        got = positive_pieces(pcs[c], npc[c])
        want = positive_pieces(r.pieces)
        diff = sym_diff_measure(got, want)
        assert diff <= 2 * max(len(want), 1) * ANG_TOL, (c, diff)
        if got.shape == want.shape:
            assert np.max(np.abs(got - want), initial=0.0) <= ANG_TOL, (c, got, want)
        assert abs(th[c] - r.theta) <= ANG_TOL, (c, th[c], r.theta)
        if rej[c]:
            np.testing.assert_array_equal(Xn[c], X[c])
        else:
            scale = 1.0 + np.abs(r.x_next)
            assert np.all(np.abs(Xn[c] - r.x_next) <= ANG_TOL * scale * (1 + np.abs(NU[c]))), c
    n_exempt = int(exempt.sum())
    assert n_exempt <= max_exempt_frac * len(idx), (n_exempt, len(idx))
    return stats, n_exempt, len(idx)


@pytest.mark.parametrize("d,m,n", [(2, 4, 16), (10, 20, 64), (37, 75, 130), (137, 300, 200),
                                   (100, 200, 256)])
def test_mixed_step_parity(d, m, n):
    rng = np.random.default_rng(31 * d + m)
    A, b, X, NU = grid_instance(rng, d, m, n, scale=1.0 / math.sqrt(d), slack=(0.05, 0.6))
    U = rng.uniform(size=n)
    check_mixed(A, b, X, NU, U)


def test_mixed_full_size_sampled():
    """d = 1000, m = 2000, 8192 chains (the benchmark's launch): the metric
    workload's rows on a grid, 64 sampled chains compared element by element."""
    import workloads
    inst = workloads.metric(n_chains=1)
    d = inst.d
    B = grid_bits(d)
    A = to_grid(inst.A, B)
    rng = np.random.default_rng(2)
    X = to_grid(rng.standard_normal((8192, d)) * 0.002, B)
    NU = to_grid(rng.standard_normal((8192, d)), B)
    U = rng.uniform(size=8192)
    assert np.max(X @ A.T - inst.b) < 0.0
    idx = rng.choice(8192, size=64, replace=False)
    check_mixed(A, inst.b, X, NU, U, sample=idx, max_pieces=64)


def test_mixed_trim_keeps_interior():
    rng = np.random.default_rng(4)
    A, b, X, NU = grid_instance(rng, 20, 60, 128, scale=0.3, slack=(0.05, 0.5))
    U = rng.uniform(size=128)
    check_mixed(A, b, X, NU, U, trim_eps=1e-4)


def test_mixed_cta_kernel_probit_orthant():
    """Mixed form through the CTA-per-chain kernel (every chain), on a
    probit-style orthant where all arcs have half-width pi / 2 and are merged
    per bucket; grid inputs, every chain compared element by element."""
    rng = np.random.default_rng(8)
    k = 256
    M = rng.standard_normal((k, k))
    B = grid_bits(k)
    L = to_grid(np.linalg.cholesky(M @ M.T / k + np.eye(k)), B)
    z = to_grid(rng.standard_normal(k), B)
    f = L @ z
    assert np.all(f != 0.0)
    y = np.sign(f)
    A = -y[:, None] * L
    b = np.zeros(k)
    n = 64
    X = np.tile(z, (n, 1))
    NU = to_grid(rng.standard_normal((n, k)), B)
    U = rng.uniform(size=n)
    check_mixed(A, b, X, NU, U, sort_threads=256)


@pytest.mark.parametrize("sort_threads", [0, 256])
@pytest.mark.parametrize("half", [False, True])
def test_mixed_long_arc_union(half, sort_threads):
    """Rows with b_i <= 0 have infeasible arcs of length >= pi; for a feasible
    x any two overlap, so together they are one arc (min alpha, max beta) and
    the step keeps only the rows holding its two extremes (Sec. 3.1's I_act
    unchanged): the warp kernel (sort_threads = 0) and the CTA-per-chain
    kernel (256).  A probit-style orthant (b = 0: no arc contains another,
    so the bucket prune alone keeps every arc), and the same with half of the
    rows given b > 0 (short arcs, pruned by the union and by each other).
    Grid inputs, every chain against the oracle; few arcs reach the sort."""
    rng = np.random.default_rng(14)
    k = 256
    M = rng.standard_normal((k, k))
    B = grid_bits(k)
    L = to_grid(np.linalg.cholesky(M @ M.T / k + np.eye(k)), B)
    z = to_grid(rng.standard_normal(k), B)
    f = L @ z
    assert np.all(f != 0.0)
    A = -np.sign(f)[:, None] * L
    b = np.zeros(k)
    if half:
        b[1::2] = to_grid(rng.uniform(0.05, 0.5, size=k // 2), B)
    n = 64
    X = np.tile(z, (n, 1))
    NU = to_grid(rng.standard_normal((n, k)), B)
    U = rng.uniform(size=n)
    stats, _, _ = check_mixed(A, b, X, NU, U, sort_threads=sort_threads)
    # without the union every chain would sort (or merge) all 256 arcs
    assert stats["sort_keys"] < 32 * n, stats["sort_keys"]


@pytest.mark.parametrize("path", ["warp", "stream", "cta"])
def test_mixed_overflow_chains(path):
    """Chains that keep more arcs than a warp sorts: rows facing away from x
    with b = 2^-8 (every arc a little shorter than a half circle, none inside
    another), so each chain keeps ~300 arcs.  The warp kernel steps them at
    the end of its own CTA ("warp"), the streamed kernel lists them for the
    CTA kernel ("stream"), or the CTA kernel takes every chain ("cta"); grid
    inputs, every chain against the oracle."""
    rng = np.random.default_rng(31)
    d, m, n = 24, 320, 48
    B = grid_bits(d)
    x = to_grid(rng.standard_normal(d), B)
    A = to_grid(rng.standard_normal((m, d)) / np.sqrt(d), B)
    A[A @ x > 0] *= -1.0
    keep = A @ x < -1e-3
    A = A[keep]
    A = A[:A.shape[0] // 4 * 4]  # the streamed kernel takes m, d multiples of 4
    b = np.full(A.shape[0], 2.0**-8)
    X = np.tile(x, (n, 1))
    NU = to_grid(rng.standard_normal((n, d)), B)
    U = rng.uniform(size=n)
    cfg = {"sort_threads": 256} if path == "cta" else {}
    kind = ess.ESS_CHAIN_STREAM if path == "stream" else None
    stats, _, _ = check_mixed(A, b, X, NU, U, chain_kernel=kind, **cfg)
    # every chain kept more arcs than a warp sorts (128)
    assert stats["sort_keys"] > 128 * n


def test_mixed_near_tangent_rows_fp64_branch():
    """Rows with b / r in (1 - 1e-4, 1): the mixed form takes the arccos
    argument and the angles in FP64 (tangent_fp64 counts them).  Grid rows,
    b = r (1 - delta) in double: the small arcs around tau cut holes in a wide
    active set, and every chain must match the oracle (no exemption)."""
    rng = np.random.default_rng(12)
    d, m0, n = 12, 20, 96
    A0, b0, X1, NU1 = grid_instance(rng, d, m0, 1, scale=0.3, slack=(1.0, 2.0))
    x, nu = X1[0], NU1[0]
    B = grid_bits(d)
    extra = to_grid(rng.standard_normal((40, d)), B)
    p, q = extra @ x, extra @ nu
    r = np.hypot(p, q)
    deltas = np.array([9e-5, 5e-5, 2e-5, 1e-5, 3e-6, 1e-6, 1e-7, 1e-8, 1e-10, 1e-12])
    rows, bs = [], []
    for i in range(extra.shape[0]):
        dl = deltas[len(rows) % deltas.size]
        if p[i] / r[i] < 1.0 - 2 * dl and len(rows) < 2 * deltas.size:
            rows.append(extra[i])
            bs.append(r[i] * (1.0 - dl))
    A = np.vstack([A0, np.array(rows)])
    b = np.concatenate([b0, np.array(bs)])
    X = np.tile(x, (n, 1))
    NU = np.tile(nu, (n, 1))
    U = (np.arange(n) + 0.5) / n
    stats, n_exempt, _ = check_mixed(A, b, X, NU, U, max_exempt_frac=0.0)
    assert n_exempt == 0
    assert stats["tangent_fp64"] >= len(rows) * n


def test_mixed_near_tangent_minus_one():
    """A row with b / r in (-1, -1 + 1e-4): x_t sits just inside the
    constraint and the whole circle but a window of half-width ~sqrt(2 delta)
    around theta = 0 is infeasible (Fig. 2(d) is the limit delta = 0).  Grid
    inputs, q = 0 exactly for that row (nu has no component along it)."""
    rng = np.random.default_rng(13)
    d, m0, n = 6, 10, 64
    A0, b0, X1, NU1 = grid_instance(rng, d, m0, 1, scale=0.3, slack=(1.0, 2.0))
    x, nu = X1[0].copy(), NU1[0].copy()
    x[0], nu[0] = 0.5, 0.0
    b0 = np.maximum(b0, A0 @ x + 0.5)
    for delta in (9e-5, 1e-6, 1e-9):
        a = np.zeros(d)
        a[0] = -1.0                       # p = -x_0 = -0.5, q = 0: tau = pi
        A = np.vstack([A0, a])
        b = np.concatenate([b0, [-0.5 * (1.0 - delta)]])
        X = np.tile(x, (n, 1))
        NU = np.tile(nu, (n, 1))
        U = (np.arange(n) + 0.5) / n
        _, n_exempt, _ = check_mixed(A, b, X, NU, U, max_exempt_frac=0.0)
        assert n_exempt == 0


def _fig1_instance():
    rows = read_golden("fig1_worked_example.txt")
    x = np.array([float(v) for v in rows[0][1:]])
    nu = np.array([float(v) for v in rows[1][1:]])
    A, b = [], []
    for row in rows[2:]:
        if row[0] == "plane":
            t1, t2 = float(row[1]) * math.pi, float(row[2]) * math.pi
            tau, h = 0.5 * (t1 + t2), 0.5 * (t2 - t1)
            A.append(np.linalg.solve(np.stack([x, nu]), [math.cos(tau), math.sin(tau)]))
            b.append(math.cos(h))
    return x, nu, np.array(A), np.array(b)


def test_mixed_fig1_worked_example():
    """Fig. 1 through the mixed form.  Its rows are not on a grid, so the
    exemption bound takes the FP16x3 product bound of q and the refresh bound
    of p (plus their float roundings and that of A): no chain may be exempt."""
    x, nu, A, b = _fig1_instance()
    U = np.array([0.0, 0.1, 0.35, 0.5, 0.77, 0.999])
    X = f32(np.tile(x, (U.size, 1)))
    NU = f32(np.tile(nu, (U.size, 1)))
    A32 = f32(A)
    absA = np.abs(A)
    eps_q = (fp16x3_bound(A32, NU) + 2.0**-24 * (np.abs(NU) @ absA.T)
             + 2.0**-24 * np.abs(NU @ A.T))
    eps_p = refresh_bound(A, X) + 2.0**-23 * np.abs(X @ A.T)
    stats, n_exempt, _ = check_mixed(A, b, X, NU, U, eps_p=eps_p, eps_q=eps_q,
                                     max_exempt_frac=0.0)
    assert n_exempt == 0


def test_mixed_fig2_edge_cases():
    """Fig. 2 gallery through the mixed form (exact inputs): b / r = 1.25 and
    1 give no root, 0.5 the arc (2 pi / 3, 4 pi / 3), -1 the single point
    {0} (theta = 0, stay)."""
    x = np.array([[2.0, 0.0]])
    nu = np.array([[0.0, 1.0]])
    a = np.array([[-1.0, 0.0]])
    for b_val in (2.5, 2.0, 1.0, -2.0):
        U = np.array([0.4])
        s = ess.Sampler(a, np.array([b_val]), precision=ess.ESS_PREC_MIXED)
        try:
            Xn, th, pcs, npc, rej = s.step_with_draws(dev(x), dev(nu), dev(U), max_pieces=4)
            Xn, th, pcs, npc = host(Xn), host(th), host(pcs), host(npc)
        finally:
            s.close()
        if b_val >= 2.0:
            np.testing.assert_allclose(positive_pieces(pcs[0], npc[0]), [[0.0, 2 * math.pi]],
                                       atol=ANG_TOL)
        elif b_val == 1.0:
            np.testing.assert_allclose(positive_pieces(pcs[0], npc[0]),
                                       [[0.0, 2 * math.pi / 3], [4 * math.pi / 3, 2 * math.pi]],
                                       atol=ANG_TOL)
        else:
            assert th[0] == 0.0 and npc[0] == 0
            np.testing.assert_array_equal(Xn[0], x[0])
        _, n_exempt, _ = check_mixed(a, np.array([b_val]), x, nu, U, max_exempt_frac=0.0)
        assert n_exempt == 0
