"""Seeded synthetic instances for the linear elliptical slice sampler.

This module only builds inputs (A, b, X0 and run sizes) from numpy's
``default_rng``; it holds none of the sampler's arithmetic.  Both the CUDA
library's tests/benchmark and the CPU oracle read their inputs from here, so
the two sides see identical data without sharing any code of the method.

The paper (arXiv 2407.10449) uses only synthetic workloads: univariate
truncations (Sec. 4.1) and random polytopes A x <= b with i.i.d. Gaussian A
(Sec. 4.2).  The families below follow that recipe at the sizes of the
benchmark configurations:

* ``small``      d=10,   m=20,   A ~ N(0,1),                 b ~ U[0.5, 1.5]
* ``medium``     d=100,  m=200,  A ~ N(0,1)/sqrt(d),         b ~ U[0.2, 1.0]
* ``metric``     d=1000, m=2000, A ~ N(0,1)/sqrt(d), unit rows, b ~ U[0.05, 0.5]
* ``probit``     n=d=m=2000 probit-GP orthant posterior (whitened by App. A)
* ``batched``    512 polytopes, d ~ U{8..256}, m ~ U{d..4d}, chains ~ U{8..64}
* ``paper_hd``   the Sec. 4.2 family: A (d x d) ~ N(0,1), b = A x0 + U[0,1]^d
* the Sec. 4.1 intervals and a 2-D box for exactness checks.

X0 = 0 is strictly feasible whenever b > 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Instance:
    name: str
    A: np.ndarray            # m x d, float64, row-major
    b: np.ndarray            # m, float64
    X0: np.ndarray           # n_chains x d, float64
    n_iter: int
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.A.shape[1]

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n_chains(self) -> int:
        return self.X0.shape[0]


def _gaussian_polytope(rng, d, m, b_lo, b_hi, scale, unit_rows=False):
    A = rng.standard_normal((m, d)) * scale
    if unit_rows:
        A /= np.linalg.norm(A, axis=1, keepdims=True)
    b = rng.uniform(b_lo, b_hi, size=m)
    return np.ascontiguousarray(A), np.ascontiguousarray(b)


def small(seed=0, n_chains=16, n_iter=1000) -> Instance:
    """d=10, m=20, A iid N(0,1), b iid U[0.5, 1.5], X0 = 0."""
    rng = np.random.default_rng(seed)
    A, b = _gaussian_polytope(rng, 10, 20, 0.5, 1.5, 1.0)
    return Instance("small_d10_m20", A, b, np.zeros((n_chains, 10)), n_iter)


def medium(seed=0, n_chains=1024, n_iter=2000) -> Instance:
    """d=100, m=200, A iid N(0,1)/sqrt(d), b iid U[0.2, 1.0], X0 = 0."""
    rng = np.random.default_rng(seed)
    d, m = 100, 200
    A, b = _gaussian_polytope(rng, d, m, 0.2, 1.0, 1.0 / np.sqrt(d))
    return Instance("medium_d100_m200", A, b, np.zeros((n_chains, d)), n_iter)


def metric(seed=0, n_chains=8192, n_iter=500, d=1000, m=2000) -> Instance:
    """d=1000, m=2000, unit-norm rows of N(0,1)/sqrt(d), b iid U[0.05, 0.5]."""
    rng = np.random.default_rng(seed)
    A, b = _gaussian_polytope(rng, d, m, 0.05, 0.5, 1.0 / np.sqrt(d), unit_rows=True)
    return Instance(f"metric_d{d}_m{m}", A, b, np.zeros((n_chains, d)), n_iter)


def probit(seed=0, n=2000, n_chains=4096, n_iter=500, lengthscale=0.2, jitter=1e-6):
    """Probit-GP orthant posterior before whitening.

    Points U[0,1]^2, K = RBF(lengthscale) + jitter I, L = chol(K), z* ~ N(0, I),
    f* = L z*, y = sign(f*).  The posterior of the latent f ~ N(0, K) given
    y_i f_i >= 0 is the truncation of N(0, K) by A0 f <= 0 with
    A0 = -diag(y).  Returned: (A0, b = 0, K, L, mu = 0, X0 = z* per chain);
    L (numpy's factor) draws the labels, and a sampler may factor K itself.
    The sampler runs in whitened coordinates (App. A): A = A0 L, b' = b.
    """
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(n, 2))
    sq = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    K = np.exp(-0.5 * sq / lengthscale ** 2) + jitter * np.eye(n)
    L = np.linalg.cholesky(K)
    z = rng.standard_normal(n)
    f = L @ z
    y = np.where(f >= 0.0, 1.0, -1.0)
    A0 = np.ascontiguousarray(-np.diag(y))
    b = np.zeros(n)
    X0 = np.tile(z, (n_chains, 1))
    return dict(A0=A0, b=b, K=K, L=np.ascontiguousarray(L), mu=np.zeros(n), X0=X0,
                n_iter=n_iter, name=f"probit_n{n}")


def probit_features(seed=0, d=256, m=16384, n_chains=2048, n_iter=200) -> Instance:
    """Probit-style orthant with m observations of d features: y_i phi_i . x
    >= 0 for all i, i.e. A = -diag(y) Phi, b = 0, Phi iid N(0, 1) / sqrt(d),
    y_i = sign(phi_i . x0) for a start x0 ~ N(0, I).  Every arc then has
    half-width pi / 2 (b = 0) and none contains another, so no row drops out
    of the domination prune: the many-arc case at m well beyond d."""
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((m, d)) / np.sqrt(d)
    x0 = rng.standard_normal(d)
    y = np.sign(Phi @ x0)
    y[y == 0] = 1.0
    A = -y[:, None] * Phi
    keep = A @ x0 < 0.0
    A = np.ascontiguousarray(A[keep])
    return Instance(f"probit_features_d{d}_m{m}", A, np.zeros(A.shape[0]),
                    np.tile(x0, (n_chains, 1)), n_iter)


def rotated_box(seed=0, d=200, lo=-1.0, hi=1.5, n_chains=1, n_iter=200) -> Instance:
    """The box lo <= y_j <= hi in a random orthonormal basis Q: A = [Q; -Q],
    b = [hi 1; -lo 1] (m = 2d).  N(0, I) is rotation invariant, so its
    probability is (Phi(hi) - Phi(lo))^d exactly (meta["log_z"]): a normal
    probability with a known value at any dimension."""
    import math
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((d, d)))
    Q = Q * np.sign(np.diag(R))[None, :]
    A = np.ascontiguousarray(np.vstack([Q, -Q]))
    b = np.concatenate([np.full(d, hi), np.full(d, -lo)])
    phi = lambda x: 0.5 * math.erfc(-x / math.sqrt(2.0))
    inst = Instance(f"rotated_box_d{d}", A, b, np.zeros((n_chains, d)), n_iter)
    inst.meta["log_z"] = d * math.log(phi(hi) - phi(lo))
    return inst


def batched(seed=0, n_problems=512, n_iter=1000, d_range=(8, 256), c_range=(8, 64)):
    """Uneven batch: d ~ U{8..256}, m ~ U{d..4d}, chains ~ U{8..64} per polytope."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_problems):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        m = int(rng.integers(d, 4 * d + 1))
        c = int(rng.integers(c_range[0], c_range[1] + 1))
        A, b = _gaussian_polytope(rng, d, m, 0.1, 1.0, 1.0 / np.sqrt(d))
        out.append(Instance(f"batched_{k}", A, b, np.zeros((c, d)), n_iter))
    return out


def paper_hd(seed=0, d=1000, n_chains=1, n_iter=1000) -> Instance:
    """Sec. 4.2 family: A (d x d) iid N(0,1), x0 ~ N(0, I), b = A x0 + U[0,1]^d."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    x0 = rng.standard_normal(d)
    b = A @ x0 + rng.uniform(0.0, 1.0, size=d)
    return Instance(f"paper_hd_d{d}", A, b, np.tile(x0, (n_chains, 1)), n_iter)


def interval(lo, hi, n_chains=16384, n_iter=200, x0=None) -> Instance:
    """d = 1 truncation lo <= x <= hi written as A = [[1], [-1]], b = [hi, -lo]."""
    A = np.array([[1.0], [-1.0]])
    b = np.array([hi, -lo], dtype=np.float64)
    if x0 is None:
        x0 = 0.5 * (lo + hi) if not (lo <= 0.0 <= hi) else 0.0
    return Instance(f"interval_{lo}_{hi}", A, b, np.full((n_chains, 1), float(x0)), n_iter)


def box2(lo=(-1.0, -0.5), hi=(3.0, 1.2), n_chains=16384, n_iter=200) -> Instance:
    """d = 2 box: A = [I; -I], b = [hi, -lo]."""
    A = np.vstack([np.eye(2), -np.eye(2)])
    b = np.array([hi[0], hi[1], -lo[0], -lo[1]], dtype=np.float64)
    return Instance("box2", A, b, np.zeros((n_chains, 2)), n_iter)


def random_states(rng, n, d, scale=1.0):
    return rng.standard_normal((n, d)) * scale
