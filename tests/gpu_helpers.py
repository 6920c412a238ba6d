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
