"""FP64 CPU oracle for linear elliptical slice sampling (arXiv 2407.10449).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
reference for the CUDA library: the tests, the smoke check and the CPU
baseline of the benchmark load it; the product path never does.  It shares no
code with the CUDA library.  The arithmetic lives in ``ess_oracle.c`` (plain C,
double precision); this module compiles it with gcc on first use and wraps it
with ctypes and numpy.

Each wrapper names the part of the paper it follows:

* ``philox4x32_10``, ``rng_block``, ``draw_nu``, ``draw_u``: the random draws
  of Alg. 1 (Philox4x32-10 per Salmon et al. 2011 plus Box-Muller; the paper
  does not specify its generator).
* ``roots``: App. B and Sec. 3.2 (closed-form roots and edge cases).
* ``active_intervals``: Alg. 2 (brute-force clipping).
* ``draw_theta``: Alg. 1, "sample uniformly theta ~ I_act" (inverse CDF).
* ``step``: one iteration of Alg. 1 with given draws, with the Sec. 3.3
  trimming and rejection.
* ``run``: many independent chains (Alg. 1 loop) with the oracle's own RNG.
* ``whiten`` / ``unwhiten``: App. A.
* ``cholesky``: App. A's factor Sigma = L L^T (Cholesky-Banachiewicz).

The Philox bit stream is pinned by an independent implementation of the
published generator (triton's language library, run on the host by its
interpreter; tests/test_oracle_philox.py), bit for bit, and the draws by
statistical tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ess_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libess_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_llp = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile ess_oracle.c into a shared library (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", "-pthread",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_rng_block.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _u32p]
        lib.orc_draw_nu.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_int, _dp]
        lib.orc_draw_u.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32]
        lib.orc_draw_u.restype = ctypes.c_double
        lib.orc_roots.argtypes = [ctypes.c_double] * 3 + [_dp, _dp]
        lib.orc_roots.restype = ctypes.c_int
        lib.orc_active_intervals.argtypes = [ctypes.c_int, _dp, _dp, _ip, _dp, _dp, ctypes.c_int]
        lib.orc_active_intervals.restype = ctypes.c_int
        lib.orc_draw_theta.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double]
        lib.orc_draw_theta.restype = ctypes.c_double
        lib.orc_max_residual.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp]
        lib.orc_max_residual.restype = ctypes.c_double
        lib.orc_step.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                 ctypes.c_double, ctypes.c_double, _dp, _dp, _dp,
                                 ctypes.c_int, _ip, _dp, _ip, _dp, _dp, _ip]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_run.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64,
                                ctypes.c_uint32, ctypes.c_double, _dp, ctypes.c_int, _llp,
                                ctypes.c_int]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_whiten.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.orc_unwhiten.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.orc_cholesky.argtypes = [_dp, ctypes.c_int, _dp]
        lib.orc_cholesky.restype = ctypes.c_int
        _lib = lib
        return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


TWO_PI = 2.0 * np.pi


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function on a 4-word counter and 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def rng_block(seed, n, chain, t, problem=0, stream=0) -> np.ndarray:
    lib = _load()
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_rng_block(seed, n, chain, t, problem, stream, _ptr(out, _u32p))
    return out


def draw_nu(seed, chain, t, d, problem=0) -> np.ndarray:
    """nu ~ N(0, I_d) of chain `chain` at iteration `t` (Alg. 1)."""
    lib = _load()
    out = np.zeros(d, dtype=np.float64)
    lib.orc_draw_nu(seed, chain, t, problem, d, _ptr(out))
    return out


def draw_u(seed, chain, t, problem=0) -> float:
    """Uniform [0, 1) for the theta draw of chain `chain` at iteration `t`."""
    return float(_load().orc_draw_u(seed, chain, t, problem))


def roots(p, q, b):
    """(kind, alpha, beta): kind 1 = arc (alpha, beta) infeasible, 0 = no root,
    -1 = x provably infeasible (App. B, Sec. 3.2)."""
    lib = _load()
    a = ctypes.c_double()
    bb = ctypes.c_double()
    k = lib.orc_roots(float(p), float(q), float(b), ctypes.byref(a), ctypes.byref(bb))
    return k, a.value, bb.value


def active_intervals(alpha, beta, use=None):
    """Alg. 2 on given pairs: ascending list of (lo, hi) pieces."""
    lib = _load()
    alpha = _f64(alpha)
    beta = _f64(beta)
    m = alpha.shape[0]
    usep = None
    if use is not None:
        use = np.ascontiguousarray(use, dtype=np.int32)
        usep = _ptr(use, _ip)
    cap = 2 * m + 4
    lo = np.zeros(cap)
    hi = np.zeros(cap)
    n = lib.orc_active_intervals(m, _ptr(alpha), _ptr(beta), usep, _ptr(lo), _ptr(hi), cap)
    if n < 0:
        raise RuntimeError("active_intervals: capacity")
    return np.stack([lo[:n], hi[:n]], axis=1)


def draw_theta(pieces, u) -> float:
    lib = _load()
    pieces = _f64(pieces).reshape(-1, 2)
    lo = np.ascontiguousarray(pieces[:, 0])
    hi = np.ascontiguousarray(pieces[:, 1])
    return float(lib.orc_draw_theta(pieces.shape[0], _ptr(lo), _ptr(hi), float(u)))


def max_residual(A, b, x) -> float:
    lib = _load()
    A = _f64(A)
    b = _f64(b)
    x = _f64(x)
    m, d = A.shape
    return float(lib.orc_max_residual(_ptr(A), _ptr(b), d, m, _ptr(x)))


class StepResult:
    __slots__ = ("status", "x_next", "pieces", "theta", "rejected", "alpha", "beta", "has_root")

    def __init__(self, **kw):
        for k, v in kw.items():
            setattr(self, k, v)


def step(A, b, x, nu, u, trim_eps=0.0) -> StepResult:
    """One iteration of Alg. 1 for one chain with given nu and u."""
    lib = _load()
    A = _f64(A)
    b = _f64(b)
    x = _f64(x)
    nu = _f64(nu)
    m, d = A.shape
    cap = 2 * m + 4
    lo = np.zeros(cap)
    hi = np.zeros(cap)
    xn = np.zeros(d)
    npieces = ctypes.c_int()
    theta = ctypes.c_double()
    rej = ctypes.c_int()
    al = np.zeros(max(m, 1))
    be = np.zeros(max(m, 1))
    hr = np.zeros(max(m, 1), dtype=np.int32)
    st = lib.orc_step(_ptr(A), _ptr(b), d, m, _ptr(x), _ptr(nu), float(u), float(trim_eps),
                      _ptr(xn), _ptr(lo), _ptr(hi), cap, ctypes.byref(npieces),
                      ctypes.byref(theta), ctypes.byref(rej), _ptr(al), _ptr(be), _ptr(hr, _ip))
    n = npieces.value
    return StepResult(status=st, x_next=xn, pieces=np.stack([lo[:n], hi[:n]], axis=1),
                      theta=theta.value, rejected=bool(rej.value), alpha=al[:m], beta=be[:m],
                      has_root=hr[:m].astype(bool))


def run(A, b, X0, n_iter, seed, t0=0, chain_offset=0, problem=0, trim_eps=0.0,
        record_every=0, n_threads=None):
    """Runs independent chains (Alg. 1) from X0 (n_chains x d).

    Returns (X_final, samples or None, rejections per chain)."""
    lib = _load()
    A = _f64(A)
    b = _f64(b)
    X = np.array(X0, dtype=np.float64, order="C", copy=True)
    if X.ndim == 1:
        X = X.reshape(1, -1)
    n_chains, d = X.shape
    m = A.shape[0]
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    samples = None
    if record_every > 0:
        samples = np.zeros((n_chains, n_iter // record_every, d))
    rej = np.zeros(n_chains, dtype=np.int64)
    st = lib.orc_run(_ptr(A), _ptr(b), d, m, _ptr(X), n_chains, chain_offset, t0, n_iter,
                     seed, problem, float(trim_eps), _ptr(samples), record_every,
                     _ptr(rej, _llp), int(n_threads))
    if st != 0:
        raise RuntimeError(f"oracle run failed with status {st}")
    return X, samples, rej


def whiten(A, b, mu, L):
    """App. A: (A L, b - A mu)."""
    lib = _load()
    A = _f64(A)
    b = _f64(b)
    L = _f64(L)
    m, d = A.shape
    mu = None if mu is None else _f64(mu)
    Ao = np.zeros((m, d))
    bo = np.zeros(m)
    lib.orc_whiten(_ptr(A), _ptr(b), _ptr(mu), _ptr(L), d, m, _ptr(Ao), _ptr(bo))
    return Ao, bo


def unwhiten(L, mu, U):
    """App. A: x = L u + mu for each row u of U."""
    lib = _load()
    L = _f64(L)
    U = _f64(U)
    if U.ndim == 1:
        U = U.reshape(1, -1)
    n, d = U.shape
    mu = None if mu is None else _f64(mu)
    X = np.zeros((n, d))
    lib.orc_unwhiten(_ptr(L), _ptr(mu), d, n, _ptr(U), _ptr(X))
    return X


def cholesky(S):
    """App. A: the lower factor L with S = L L^T (only S's lower triangle is
    read).  Raises ValueError naming the row whose pivot is not positive."""
    lib = _load()
    S = _f64(S)
    n = S.shape[0]
    L = np.zeros((n, n))
    info = lib.orc_cholesky(_ptr(S), n, _ptr(L))
    if info != 0:
        raise ValueError(f"not positive definite: pivot of row {info - 1}")
    return L


# ---------------------------------------------------------------------------
# Normal probability of the domain, Z = P(A x <= b) for x ~ N(0, I) (the
# normaliser of the target of Sec. 2), by the Holmes-Diaconis-Ross (HDR)
# splitting estimator driven by the sampler -- the use the paper cites in its
# introduction and related work (Gessner et al. 2020).  The paper gives no
# algorithm for it; the steps below restate the published method:
#   nested domains D_t = {x : A x <= b + gamma_t}, gamma_1 > ... > gamma_T = 0;
#   Z = P(D_1) prod_t P(D_t | D_(t-1)), each factor estimated by the fraction
#   of n samples of the truncated normal on D_(t-1) that lie in D_t, the
#   samples of level t drawn by elliptical slice sampling on D_(t-1) started
#   from the samples of level t - 1 that lie in D_(t-1) ("splitting").
# The shifts come from a first stage (subset simulation): gamma_t sits
# between the k-th and (k+1)-th smallest level values, k = ceil(rho n), so
# that a fraction rho of the samples falls in each next domain; the second
# stage (HDR proper) repeats the levels with fresh draws at those fixed shifts.
# Random numbers: the start samples of a stage are Philox normals of (seed,
# chain j, t = 0, problem 1); level t's chains take the steps (t - 1) k_b ..
# t k_b - 1 of run() with problem 0, k_b = n_between.  Stage 1 uses seed,
# stage 2 seed + 1.
# ---------------------------------------------------------------------------

def hdr_level(A, b, X):
    """g(x) = max_i (a_i . x - b_i) per row of X: x lies in {A x <= b + gamma}
    exactly when g(x) <= gamma."""
    return np.max(np.asarray(X) @ _f64(A).T - _f64(b)[None, :], axis=1)


def hdr_start(seed, n, d):
    """The n start samples of a stage: independent N(0, I_d) draws."""
    return np.stack([draw_nu(seed, j, 0, d, problem=1) for j in range(n)])


def hdr_stage(A, b, n_samples, rho, n_between, seed, shifts=None, max_levels=64):
    """One stage of the estimator; returns (shifts, counts) per level.

    shifts None: subset simulation -- level t's shift is the midpoint of the
    k-th and (k + 1)-th smallest g over the level's samples (k = ceil(rho n)),
    or 0 once the k-th smallest is <= 0 (the last level).  Otherwise the given
    shifts (the last must be 0) are used in turn; a level with no sample
    inside ends the stage (Z estimate 0)."""
    A = _f64(A)
    b = _f64(b)
    m, d = A.shape
    n = int(n_samples)
    k = int(np.ceil(rho * n))
    if not (1 <= k <= n - 1):
        raise ValueError("need 1 <= ceil(rho n) <= n - 1")
    X = hdr_start(seed, n, d)
    out_shifts, counts = [], []
    while True:
        level = len(out_shifts)
        g = hdr_level(A, b, X)
        if shifts is None:
            gs = np.sort(g)
            gamma = 0.0 if gs[k - 1] <= 0.0 else gs[k - 1] + (gs[k] - gs[k - 1]) / 2.0
        else:
            gamma = float(shifts[level])
        inside = g <= gamma
        cnt = int(inside.sum())
        out_shifts.append(gamma)
        counts.append(cnt)
        if gamma == 0.0 or cnt == 0:
            break
        if len(out_shifts) >= max_levels:
            raise RuntimeError("no level reached the domain within max_levels")
        seeds = X[inside]
        X0 = seeds[np.arange(n) % cnt]
        X = run(A, b + gamma, X0, n_between, seed, t0=level * n_between)[0]
    return np.array(out_shifts), np.array(counts)


def hdr(A, b, n_samples, rho=0.5, n_between=8, seed=0, max_levels=64):
    """Z = P(A x <= b), x ~ N(0, I): subset simulation for the shifts, then
    HDR at those shifts.  Returns a dict with log_z (HDR), the shifts and
    per-level counts of both stages, and log_z_ss (the subset-simulation
    estimate of stage 1)."""
    s1, c1 = hdr_stage(A, b, n_samples, rho, n_between, seed, None, max_levels)
    s2, c2 = hdr_stage(A, b, n_samples, rho, n_between, seed + 1, s1, max_levels)
    n = float(n_samples)
    with np.errstate(divide="ignore"):
        log_z = float(np.sum(np.log(c2 / n))) if len(c2) == len(s1) else -np.inf
        log_z_ss = float(np.sum(np.log(c1 / n)))
    return dict(log_z=log_z, shifts=s1, counts=c2, counts_ss=c1, log_z_ss=log_z_ss)
