"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import math

import numpy as np

import oracle

TWO_PI = 2.0 * math.pi


def dev(a, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def positive_pieces(pieces, n=None):
    """Pieces of positive length, as a (k, 2) array."""
    p = np.asarray(pieces, dtype=np.float64).reshape(-1, 2)
    if n is not None:
        p = p[:n]
    return p[p[:, 1] > p[:, 0]]


def merge(pieces, tol=0.0):
    """Union of pieces as disjoint intervals (pieces closer than tol are joined)."""
    out = []
    for lo, hi in sorted(map(tuple, np.asarray(pieces).reshape(-1, 2))):
        if hi < lo:
            continue
        if out and lo <= out[-1][1] + tol:
            out[-1][1] = max(out[-1][1], hi)
        else:
            out.append([lo, hi])
    return np.array(out).reshape(-1, 2)


def measure(p):
    p = np.asarray(p).reshape(-1, 2)
    return float(np.sum(np.maximum(p[:, 1] - p[:, 0], 0.0)))


def sym_diff_measure(p1, p2):
    """|P1 symmetric-difference P2| for two unions of closed intervals."""
    a, b = merge(p1), merge(p2)
    pts = sorted(set(a.ravel().tolist()) | set(b.ravel().tolist()))
    total = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        mid = 0.5 * (lo + hi)
        in_a = any(l <= mid <= h for l, h in a)
        in_b = any(l <= mid <= h for l, h in b)
        if in_a != in_b:
            total += hi - lo
    return total


def oracle_steps(A, b, X, NU, U, trim_eps=0.0):
    return [oracle.step(A, b, X[c], NU[c], float(U[c]), trim_eps) for c in range(X.shape[0])]


def feasible_instance(rng, d, m, n_chains, scale=1.0, slack=(0.0, 1.0)):
    """Random polytope with strictly feasible random start points (one x per chain)."""
    A = rng.standard_normal((m, d)) * scale
    X = rng.standard_normal((n_chains, d)) * 0.3
    b = (X @ A.T).max(axis=0) + rng.uniform(*slack, size=m)
    return A, b, X


def fp16x3_bound(A, NU):
    """Bound on |q - a.nu| per chain (row of NU) and row of A for the scaled
    FP16x3 products: row i of A (rounded to float) is scaled by s_i so that its
    largest entry lies in [2^14, 2^15), chain c of nu by t_c likewise (or by
    2^12 for drawn nu), each split as v = h0 + h1 + r with fp16 h0, h1:
    |r| <= 2^-22 |v| + 2^-25 (the second term when h1 is subnormal).  The two
    residuals and the dropped h1.a1 product give 12 x 2^-24 relative to
    |a||nu|; the FP32 accumulation over K/16 tensor-core steps and the final
    addition of the two accumulators add K/16 + 2.  Unscaled, the subnormal
    terms are below 2^-38 max|nu_c| per |a_j| and 2^-38 max|a_i| per |nu_j|."""
    absdot = np.abs(NU) @ np.abs(A).T
    k = A.shape[1]
    sub = 2.0**-38 * (np.abs(NU).max(axis=1)[:, None] * np.abs(A).sum(axis=1)[None, :]
                      + np.abs(NU).sum(axis=1)[:, None] * np.abs(A).max(axis=1)[None, :])
    return absdot * (16 + k / 16) * 2.0**-24 + sub


def f32(a):
    """Values rounded to float (as the mixed form stores its inputs)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def grid_bits(d):
    """Largest B with d (2^B - 1)^2 < 2^24 (at most 11, fp16's significand)."""
    B = 11
    while B > 1 and d * (2**B - 1) ** 2 >= 2**24:
        B -= 1
    return B


def to_grid(V, B):
    """V rounded to integer multiples k 2^-e of one power of two, |k| <= 2^B - 1
    (e chosen from max |V|)."""
    V = np.asarray(V, dtype=np.float64)
    mx = float(np.abs(V).max()) if V.size else 0.0
    if mx == 0.0:
        return V.copy()
    e = math.floor(math.log2((2**B - 1) / mx))
    k = np.clip(np.round(V * 2.0**e), -(2**B - 1), 2**B - 1)
    return k * 2.0**-e


def grid_instance(rng, d, m, n_chains, scale=1.0, slack=(0.0, 1.0), x_scale=0.3):
    """Random polytope whose A, start points X and directions NU lie on grids
    on which the mixed form's products are exact.

    Each of A, X, NU holds integers k 2^-e (one power of two per array) with
    |k| <= 2^B - 1 and d (2^B - 1)^2 < 2^24.  Then every product a_i.x and
    a_i.nu is an integer multiple of one power of two below 2^24 of those
    units, so every partial sum is a float: the FP32 accumulation is exact in
    any order.  The operands survive the kernels' power-of-two scalings and
    splits exactly: after the FP16x3 GEMM scales a row (or a chain's nu) so
    that its largest entry lies in [2^14, 2^15), every entry is an integer of
    at most B <= 11 bits times a power of two >= 8, an fp16 value (the second
    slice is zero); the refresh scales x (and a row) by a power of two
    t >= max |x| and cuts x / t into w-bit slices, and x / t has at most
    B + 1 fractional bits, within the 35 (mixed) or 56 (FP64 split) bits it
    keeps.  So P and Q carry no product error; b is an arbitrary double."""
    B = grid_bits(d)
    A = to_grid(rng.standard_normal((m, d)) * scale, B)
    X = to_grid(rng.standard_normal((n_chains, d)) * x_scale, B)
    NU = to_grid(rng.standard_normal((n_chains, d)), B)
    b = (X @ A.T).max(axis=0) + rng.uniform(*slack, size=m)
    return A, b, X, NU


def long_arc_instance(rng, d, n_chains, kind, extra_rows=0, grid=False):
    """A polytope with rows of b_i <= 0, whose infeasible arcs are at least a
    half circle long (Sec. 3.1): the probit-style orthant {x : -sign(f_i)
    (L x)_i <= 0} around z, with f = L z and L = chol(M M^T / d + I)
    ("orthant": b = 0, no arc inside another); the same with b_i in
    [0.05, 0.5] on every other row ("half"); b_i = -|f_i| / 2 < 0 on every
    other row and b_i in [0.05, 0.5] on the rest ("negative").  extra_rows
    random rows with b = a.z + U[0.1, 1] follow.  Every chain starts at z,
    strictly inside.  grid: A, z and NU on the grids of grid_instance (exact
    mixed-form products); b is any double.  Returns A, b, X, NU."""
    B = grid_bits(d)
    M = rng.standard_normal((d, d))
    L = np.linalg.cholesky(M @ M.T / d + np.eye(d))
    z = rng.standard_normal(d)
    if grid:
        L, z = to_grid(L, B), to_grid(z, B)
    f = L @ z
    assert np.all(f != 0.0)
    A = -np.sign(f)[:, None] * L
    b = np.zeros(d)
    if kind in ("half", "negative"):
        b[1::2] = rng.uniform(0.05, 0.5, size=d // 2)
    if kind == "negative":
        b[0::2] = -0.5 * np.abs(f[0::2])
    if extra_rows:
        E = rng.standard_normal((extra_rows, d)) / math.sqrt(d)
        if grid:
            E = to_grid(E, B)
        A = np.vstack([A, E])
        b = np.concatenate([b, E @ z + rng.uniform(0.1, 1.0, size=extra_rows)])
    X = np.tile(z, (n_chains, 1))
    NU = rng.standard_normal((n_chains, d))
    if grid:
        NU = to_grid(NU, B)
    assert np.all(X @ A.T - b[None, :] < 0.0)
    return A, b, X, NU


# Error of the FP32 root arithmetic of the mixed form (atan2f 3 ulp, acosf 2
# ulp, the 2 pi shift and the subtraction tau - h, each at most 2^-21 rad per
# ulp for angles below 2 pi), and of the float rounding of an FP64 root.
ARITH_F32 = 7 * 2.0**-21
ARITH_F64 = 2.0**-22
# Relative error of the float ratio b / r: b rounded to float, r^2 by one
# fused multiply-add after a rounded product, the square root and the division.
RATIO_F32 = 4 * 2.0**-24


def mixed_endpoint_bounds(A, b, X, NU, eps_p=0.0, eps_q=0.0, thresh=1e-4):
    """A-priori bounds per chain (row of X, NU) and row of A on the movement
    of the mixed form's arc endpoints tau -+ h (App. B) against the exact
    FP64 roots, computed from the inputs only.

    eps_p, eps_q: bounds on the errors of the products p = A x and q = A nu
    (zero on grid inputs).  The product error moves the point (p, q) by at
    most delta = hypot(eps_p, eps_q): tau by arcsin(delta / r) and r by delta.
    The ratio b / r then moves by (eps_b + |b| delta / r) / (r - delta), plus
    RATIO_F32 |b / r| where the kernel takes it in FP32 (|b / r| <= 1 - thresh;
    beyond that the ratio and the arccos are taken in FP64 from b's double),
    and h = arccos(b / r) by the largest change of arccos over that range.
    Returns (amp, arith): the conditioning-amplified part and the fixed
    arithmetic part."""
    p = X @ A.T
    q = NU @ A.T
    r = np.hypot(p, q)
    delta = np.hypot(eps_p, eps_q) * np.ones_like(r)
    bb = np.broadcast_to(b[None, :], r.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = bb / r
        # the kernel's branch test is taken on the float ratio: rows within its
        # rounding of the threshold may take either branch (the FP32 one bounds both)
        fp32 = np.abs(ratio) <= 1.0 - thresh + 2 * RATIO_F32
        eps_b = np.where(fp32, 2.0**-24 * np.abs(bb), 0.0)
        dtau = np.arcsin(np.minimum(1.0, delta / r))
        dratio = (eps_b + np.abs(bb) * delta / r) / np.maximum(r - delta, 0.0)
        dratio = dratio + np.where(fp32, RATIO_F32 * np.abs(ratio), 0.0)
        rc = np.clip(ratio, -1.0, 1.0)
        h = np.arccos(rc)
        dh = np.maximum(np.abs(np.arccos(np.clip(rc - dratio, -1, 1)) - h),
                        np.abs(np.arccos(np.clip(rc + dratio, -1, 1)) - h))
        amp = dtau + dh
    amp = np.where(np.isfinite(amp), amp, np.inf)
    arith = np.where(fp32, ARITH_F32, ARITH_F64)
    return amp, arith


def mixed_exempt(refs, amp, arith, limit, trim_eps=0.0):
    """Per chain: True if an arc endpoint that can reach an endpoint of the
    oracle's active pieces has a conditioning bound above `limit`.  The union
    of the arcs moves only where an arc endpoint, moved within its bound,
    reaches one of the union's endpoints; rows without roots (b / r >= 1)
    gain no arc on grid inputs, since the kernel decides |b / r| within
    thresh of 1 in FP64."""
    out = np.zeros(len(refs), dtype=bool)
    for c, r in enumerate(refs):
        ends = positive_pieces(r.pieces).ravel()
        ends = ends[(ends > 0.0) & (ends < TWO_PI)]
        if ends.size == 0:
            continue
        rows = np.flatnonzero(r.has_root)
        reach = amp[c, rows] + arith[c, rows] + trim_eps + 1e-12
        da = np.abs(r.alpha[rows, None] - ends[None, :]).min(axis=1)
        db = np.abs(r.beta[rows, None] - ends[None, :]).min(axis=1)
        near = (np.minimum(da, db) <= reach)
        out[c] = bool(np.any(near & (amp[c, rows] > limit)))
    return out
