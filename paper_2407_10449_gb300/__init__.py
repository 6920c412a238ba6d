"""Python binding of the GB300 linear elliptical slice sampler (C ABI in include/ess.h).

Argument marshalling only: every step of the sampler runs in the CUDA
kernels of ``libess_gb300.so``.  Device buffers are torch CUDA tensors, passed
by pointer; streams are torch streams.  The library is built in-tree with
``paper_2407_10449_gb300.build``; if it is missing, loading fails loudly --
there is no CPU path.

The names mirror the C entry points (``ess_create``, ``ess_run``,
``ess_step_with_draws``, ...).  ``Sampler`` is a thin object wrapper.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ESS_OK = 0
ESS_ERR_ARG = 1
ESS_ERR_INFEASIBLE_X0 = 2
ESS_ERR_CUDA = 3
ESS_ERR_NUMERIC = 4
ESS_ERR_TIMEOUT = 5
ESS_ERR_OOM = 6
ESS_ERR_UNSUPPORTED = 7

ESS_PREC_FP64 = 0
ESS_PREC_MIXED = 1
ESS_REFRESH_FP64 = 0
ESS_REFRESH_SPLIT = 1
ESS_PRODUCTS_DFMA = 0
ESS_PRODUCTS_SPLIT = 1

_STATUS_NAMES = {0: "ESS_OK", 1: "ESS_ERR_ARG", 2: "ESS_ERR_INFEASIBLE_X0", 3: "ESS_ERR_CUDA",
                 4: "ESS_ERR_NUMERIC", 5: "ESS_ERR_TIMEOUT", 6: "ESS_ERR_OOM",
                 7: "ESS_ERR_UNSUPPORTED"}

# every symbol include/ess.h declares
EXPORTED = ("ess_default_config", "ess_create", "ess_destroy", "ess_limits", "ess_run",
            "ess_chains_init", "ess_chains_step", "ess_chains_get", "ess_run_host", "ess_run_few", "ess_step_with_draws", "ess_products", "ess_philox_blocks",
            "ess_draw_normals",
            "ess_set_timing", "ess_get_timing", "ess_reset_timing",
            "ess_get_stats", "ess_reset_stats", "ess_whiten", "ess_unwhiten", "ess_step_noalloc",
            "ess_cholesky", "ess_selftest_wait", "ess_hdr",
            "ess_set_graphs", "ess_graph_launches", "ess_get_tuning",
            "ess_set_chain_kernel", "ess_get_chain_kernel",
            "ess_whitener_create", "ess_whitener_destroy", "ess_whitener_apply",
            "ess_batch_create", "ess_batch_destroy", "ess_batch_run", "ess_batch_step_with_draws",
            "ess_batch_products", "ess_batch_get_stats", "ess_batch_reset_stats",
            "ess_batch_set_graphs", "ess_batch_set_persistent", "ess_batch_set_timing", "ess_batch_get_timing",
            "ess_batch_reset_timing", "ess_batch_info", "ess_batch_selftest_wait",
            "ess_last_error")

NOALLOC_SCRATCH_BYTES = 16 << 20

PHASES = ("draw", "gemm", "chain", "refresh")


class EssError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ess_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("refresh_k", ctypes.c_int),
                ("refresh_mode", ctypes.c_int), ("tangent_thresh", ctypes.c_double),
                ("trim_eps", ctypes.c_double), ("residual_margin", ctypes.c_double),
                ("sort_threads", ctypes.c_int), ("autotune", ctypes.c_int),
                ("q_tile", ctypes.c_int), ("fp64_products", ctypes.c_int),
                ("wait_limit_us", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class ess_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("rejections", ctypes.c_longlong),
                ("residual_rechecks", ctypes.c_longlong), ("tangent_fp64", ctypes.c_longlong),
                ("max_refresh_drift", ctypes.c_double), ("max_residual", ctypes.c_double),
                ("numeric_errors", ctypes.c_longlong), ("sort_keys", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Loads libess_gb300.so (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it with "
                               "paper_2407_10449_gb300.build.build()")
        lib = ctypes.CDLL(path)
        c_int, c_u64, c_u32 = ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32
        sig = {
            "ess_default_config": ([c_int, ctypes.POINTER(ess_config)], c_int),
            "ess_create": ([_dp, _dp, c_int, c_int, ctypes.POINTER(ess_config),
                            ctypes.POINTER(_vp)], c_int),
            "ess_destroy": ([_vp], None),
            "ess_limits": ([_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)], c_int),
            "ess_run": ([_vp, _vp, c_int, c_int, c_int, c_u64, _vp, c_int, _vp], c_int),
            "ess_chains_init": ([_vp, _vp, c_int, c_int, _vp], c_int),
            "ess_chains_step": ([_vp, c_int, c_u64, _vp, c_int, _vp], c_int),
            "ess_chains_get": ([_vp, _vp, _vp], c_int),
            "ess_run_host": ([_vp, _vp, c_int, c_int, c_int, c_u64, _vp, c_int, _vp], c_int),
            "ess_run_few": ([_vp, _vp, c_int, c_int, c_int, c_u64, _vp, c_int, _vp], c_int),
            "ess_cholesky": ([_vp, c_int, c_int, ctypes.POINTER(c_int), _vp], c_int),
            "ess_selftest_wait": ([_vp], c_int),
            "ess_hdr": ([_vp, c_int, ctypes.c_double, c_int, c_u64, c_int, _vp, _vp, _vp,
                         ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double), _vp], c_int),
            "ess_step_with_draws": ([_vp, _vp, _vp, _vp, c_int, _vp, _vp, _vp, c_int, _vp, _vp,
                                     _vp], c_int),
            "ess_products": ([_vp, _vp, _vp, c_int, _vp, _vp, _vp], c_int),
            "ess_philox_blocks": ([c_u64, c_u32, c_u32, c_u32, c_u32, c_int, _vp, _vp], c_int),
            "ess_draw_normals": ([_vp, c_int, c_int, c_u64, _vp, _vp], c_int),
            "ess_set_timing": ([_vp, c_int], c_int),
            "ess_get_timing": ([_vp, _vp, _vp, c_int], c_int),
            "ess_reset_timing": ([_vp], c_int),
            "ess_get_stats": ([_vp, ctypes.POINTER(ess_stats)], c_int),
            "ess_reset_stats": ([_vp], c_int),
            "ess_whiten": ([_dp, _dp, _dp, _dp, c_int, c_int, _dp, _dp], c_int),
            "ess_unwhiten": ([_dp, _dp, c_int, c_int, _dp, _dp], c_int),
            "ess_step_noalloc": ([_vp, _vp, c_int, c_int, _vp, _vp, _vp, c_int, _vp, _vp, _vp,
                                  _vp], c_int),
            "ess_whitener_create": ([_dp, _dp, c_int, ctypes.POINTER(_vp)], c_int),
            "ess_whitener_destroy": ([_vp], None),
            "ess_whitener_apply": ([_vp, _vp, c_int, c_int, _vp, _vp], c_int),
            "ess_set_graphs": ([_vp, c_int], c_int),
            "ess_set_chain_kernel": ([_vp, c_int], c_int),
            "ess_get_chain_kernel": ([_vp, ctypes.POINTER(c_int)], c_int),
            "ess_get_tuning": ([_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)], c_int),
            "ess_graph_launches": ([_vp, ctypes.POINTER(ctypes.c_longlong)], c_int),
            "ess_batch_create": ([c_int, _vp, _vp, _dp, _dp, ctypes.POINTER(ess_config),
                                  ctypes.POINTER(_vp)], c_int),
            "ess_batch_destroy": ([_vp], None),
            "ess_batch_run": ([_vp, _vp, _vp, c_int, c_int, c_u64, _vp, c_int, _vp], c_int),
            "ess_batch_step_with_draws": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], c_int),
            "ess_batch_products": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp], c_int),
            "ess_batch_get_stats": ([_vp, ctypes.POINTER(ess_stats)], c_int),
            "ess_batch_reset_stats": ([_vp], c_int),
            "ess_batch_set_graphs": ([_vp, c_int], c_int),
            "ess_batch_set_persistent": ([_vp, c_int], c_int),
            "ess_batch_set_timing": ([_vp, c_int], c_int),
            "ess_batch_get_timing": ([_vp, _vp, _vp, c_int], c_int),
            "ess_batch_reset_timing": ([_vp], c_int),
            "ess_batch_info": ([_vp, _vp, _vp, _vp, _vp], c_int),
            "ess_batch_selftest_wait": ([_vp, _vp, _vp], c_int),
            "ess_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status):
    if status != ESS_OK:
        msg = load().ess_last_error()
        raise EssError(status, msg.decode() if msg else "")


def _ptr(t):
    """Device/host pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _np64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------- C names --

def ess_default_config(precision=ESS_PREC_FP64) -> ess_config:
    cfg = ess_config()
    _check(load().ess_default_config(precision, ctypes.byref(cfg)))
    return cfg


def ess_create(A, b, cfg: ess_config | None = None):
    A = _np64(A)
    b = _np64(b)
    m, d = A.shape
    st = _vp()
    _check(load().ess_create(A.ctypes.data_as(_dp), b.ctypes.data_as(_dp), d, m,
                             ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(st)))
    return st


def ess_destroy(state):
    load().ess_destroy(state)


def ess_limits(state):
    mm, md = ctypes.c_int(), ctypes.c_int()
    _check(load().ess_limits(state, ctypes.byref(mm), ctypes.byref(md)))
    return mm.value, md.value


def ess_run(state, X, n_chains, t0, n_iter, seed, samples=None, record_every=0, stream=None):
    _check(load().ess_run(state, _ptr(X), n_chains, t0, n_iter, seed, _ptr(samples), record_every,
                          _stream_ptr(stream)))


def ess_chains_init(state, X, n_chains, t0=0, stream=None):
    _check(load().ess_chains_init(state, _ptr(X), n_chains, t0, _stream_ptr(stream)))


def ess_chains_step(state, n_iter, seed, samples=None, record_every=0, stream=None):
    _check(load().ess_chains_step(state, n_iter, seed, _ptr(samples), record_every,
                                  _stream_ptr(stream)))


def ess_chains_get(state, X=None, stream=None):
    _check(load().ess_chains_get(state, _ptr(X), _stream_ptr(stream)))


def ess_run_few(state, X, n_chains, t0, n_iter, seed, samples=None, record_every=0, stream=None):
    """1 to 16 FP64 chains, all steps in one persistent kernel (see include/ess.h).
    X: CUDA float64 (n_chains, d), updated in place; samples: CUDA float64
    (n_chains, n_iter // record_every, d) or None."""
    _check(load().ess_run_few(state, _ptr(X), n_chains, t0, n_iter, seed, _ptr(samples),
                              record_every, _stream_ptr(stream)))


def ess_run_host(state, X, n_chains, t0, n_iter, seed, samples=None, record_every=0, stream=None):
    _check(load().ess_run_host(state, _ptr(X), n_chains, t0, n_iter, seed, _ptr(samples),
                               record_every, _stream_ptr(stream)))


def ess_step_with_draws(state, X, nu, u, n_chains, X_next, theta=None, pieces=None, max_pieces=0,
                        n_pieces=None, rejected=None, stream=None):
    _check(load().ess_step_with_draws(state, _ptr(X), _ptr(nu), _ptr(u), n_chains, _ptr(X_next),
                                      _ptr(theta), _ptr(pieces), max_pieces, _ptr(n_pieces),
                                      _ptr(rejected), _stream_ptr(stream)))


def ess_products(state, X, nu, n_chains, P=None, Q=None, stream=None):
    _check(load().ess_products(state, _ptr(X), _ptr(nu), n_chains, _ptr(P), _ptr(Q),
                               _stream_ptr(stream)))


def ess_philox_blocks(seed, chain, t, problem, stream_id, n_blocks, out, stream=None):
    _check(load().ess_philox_blocks(seed, chain, t, problem, stream_id, n_blocks, _ptr(out),
                                    _stream_ptr(stream)))


def ess_draw_normals(state, n_chains, t, seed, out, stream=None):
    _check(load().ess_draw_normals(state, n_chains, t, seed, _ptr(out), _stream_ptr(stream)))


def ess_set_timing(state, enable=True):
    _check(load().ess_set_timing(state, 1 if enable else 0))


def ess_get_timing(state) -> dict:
    ms = np.zeros(len(PHASES), dtype=np.float64)
    n = np.zeros(len(PHASES), dtype=np.int64)
    _check(load().ess_get_timing(state, ms.ctypes.data, n.ctypes.data, len(PHASES)))
    return {p: {"ms": float(ms[i]), "launches": int(n[i])} for i, p in enumerate(PHASES)}


def ess_reset_timing(state):
    _check(load().ess_reset_timing(state))


def ess_get_stats(state) -> dict:
    s = ess_stats()
    _check(load().ess_get_stats(state, ctypes.byref(s)))
    return s.as_dict()


def ess_reset_stats(state):
    _check(load().ess_reset_stats(state))


def ess_whiten(A, b, mu, L):
    A = _np64(A)
    b = _np64(b)
    L = _np64(L)
    m, d = A.shape
    mu_p = None if mu is None else _np64(mu)
    A_out = np.zeros((m, d))
    b_out = np.zeros(m)
    _check(load().ess_whiten(A.ctypes.data_as(_dp), b.ctypes.data_as(_dp),
                             None if mu_p is None else mu_p.ctypes.data_as(_dp),
                             L.ctypes.data_as(_dp), d, m, A_out.ctypes.data_as(_dp),
                             b_out.ctypes.data_as(_dp)))
    return A_out, b_out


def ess_unwhiten(L, mu, U):
    L = _np64(L)
    U = _np64(U)
    if U.ndim == 1:
        U = U.reshape(1, -1)
    n, d = U.shape
    mu_p = None if mu is None else _np64(mu)
    X = np.zeros((n, d))
    _check(load().ess_unwhiten(L.ctypes.data_as(_dp),
                               None if mu_p is None else mu_p.ctypes.data_as(_dp), d, n,
                               U.ctypes.data_as(_dp), X.ctypes.data_as(_dp)))
    return X


def ess_step_noalloc(A, b, X, nu, u, X_next, theta=None, rejected=None, stream=None):
    """FP64 one-step map without any device allocation (see include/ess.h).

    For callers that may not allocate device memory at call time (a host
    framework owning the memory budget, an allocation-free request path).
    A (m, d), b (m,), X, nu, X_next (n, d), u (n,) and the optional theta (n,)
    and rejected (n, int32) are contiguous float64 CUDA tensors on one device;
    scratch comes from a fixed 16 MiB array inside the library, so calls must
    not overlap on the GPU.  Synchronous."""
    import torch
    if A.dim() != 2:
        raise ValueError("A must be (m, d)")
    m, d = A.shape
    n = X.shape[0] if X.dim() == 2 else -1
    want = [("A", A, (m, d)), ("b", b, (m,)), ("X", X, (n, d)), ("nu", nu, (n, d)),
            ("u", u, (n,)), ("X_next", X_next, (n, d))]
    if theta is not None:
        want.append(("theta", theta, (n,)))
    if rejected is not None:
        want.append(("rejected", rejected, (n,)))
    devices = set()
    for name, t, shape in want:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        dtype = torch.int32 if name == "rejected" else torch.float64
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}")
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {shape}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        devices.add(t.device)
    if len(devices) != 1:
        raise ValueError("all tensors must be on one device")
    with torch.cuda.device(devices.pop()):
        _check(load().ess_step_noalloc(_ptr(A), _ptr(b), d, m, _ptr(X), _ptr(nu), _ptr(u), n,
                                       _ptr(X_next), _ptr(theta), _ptr(rejected),
                                       _stream_ptr(stream)))


def ess_selftest_wait(state):
    """Bounded-wait self-test (see include/ess.h): raises EssError with
    ESS_ERR_TIMEOUT when the waits gave up as they should."""
    _check(load().ess_selftest_wait(state))


def ess_hdr(state, n_samples, rho=0.5, n_between=8, seed=0, max_levels=256, stream=None):
    """Normal probability P(A x <= b), x ~ N(0, I), of the state's polytope by
    the HDR splitting estimator (see include/ess.h).  Returns a dict: log_z
    (HDR), log_z_ss (subset simulation), shifts, counts, counts_ss."""
    shifts = np.zeros(max_levels)
    counts = np.zeros(max_levels, dtype=np.int32)
    counts_ss = np.zeros(max_levels, dtype=np.int32)
    nl = ctypes.c_int()
    lz, lzs = ctypes.c_double(), ctypes.c_double()
    _check(load().ess_hdr(state, int(n_samples), float(rho), int(n_between), int(seed),
                          int(max_levels), shifts.ctypes.data, counts.ctypes.data,
                          counts_ss.ctypes.data, ctypes.byref(nl), ctypes.byref(lz),
                          ctypes.byref(lzs), _stream_ptr(stream)))
    T = nl.value
    return dict(log_z=lz.value, log_z_ss=lzs.value, shifts=shifts[:T].copy(),
                counts=counts[:T].copy(), counts_ss=counts_ss[:T].copy())


def ess_cholesky(A, stream=None):
    """In place: the lower triangle of the CUDA float64 (n, n) tensor A becomes
    its Cholesky factor L (see include/ess.h).  Returns A."""
    import torch
    if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dtype == torch.float64 and A.dim() == 2
            and A.shape[0] == A.shape[1] and A.stride(1) == 1):
        raise ValueError("A must be a square CUDA float64 tensor with contiguous rows")
    info = ctypes.c_int()
    with torch.cuda.device(A.device):
        _check(load().ess_cholesky(_ptr(A), A.shape[0], A.stride(0), ctypes.byref(info),
                                   _stream_ptr(stream)))
    return A


def cholesky(S):
    """Lower Cholesky factor of S (numpy or CUDA tensor) on the GPU, as a new
    CUDA float64 tensor with zeros above the diagonal."""
    import torch
    A = torch.as_tensor(np.ascontiguousarray(S, dtype=np.float64) if isinstance(S, np.ndarray)
                        else S, dtype=torch.float64).to("cuda").contiguous().clone()
    ess_cholesky(A)
    return torch.tril(A)


def ess_whitener_create(L, mu=None):
    L = _np64(L)
    d = L.shape[0]
    mu_p = None if mu is None else _np64(mu)
    w = _vp()
    _check(load().ess_whitener_create(L.ctypes.data_as(_dp),
                                      None if mu_p is None else mu_p.ctypes.data_as(_dp), d,
                                      ctypes.byref(w)))
    return w


def ess_whitener_destroy(w):
    load().ess_whitener_destroy(w)


def ess_whitener_apply(w, U, X, stream=None):
    """X = U L^T + mu for CUDA tensors U, X (n x d, both float32 or both float64)."""
    import torch
    u_double = 1 if U.dtype == torch.float64 else 0
    if X.dtype != U.dtype:
        raise ValueError("U and X must have the same dtype")
    n = U.shape[0] if U.dim() > 1 else 1
    _check(load().ess_whitener_apply(w, _ptr(U), u_double, n, _ptr(X), _stream_ptr(stream)))


class Whitener:
    """x = L u + mu on the GPU (App. A) for batches of samples."""

    def __init__(self, L, mu=None):
        self.L = _np64(L)
        self.d = self.L.shape[0]
        self._w = ess_whitener_create(self.L, mu)

    def close(self):
        if self._w is not None:
            ess_whitener_destroy(self._w)
            self._w = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __call__(self, U, stream=None):
        import torch
        U = U.reshape(-1, self.d).contiguous()
        X = torch.empty_like(U)
        ess_whitener_apply(self._w, U, X, stream)
        return X


ESS_CHAIN_AUTO = 0
ESS_CHAIN_WARP = 1
ESS_CHAIN_STREAM = 2
ESS_CHAIN_CTA = 3


def ess_set_chain_kernel(state, kind):
    _check(load().ess_set_chain_kernel(state, int(kind)))


def ess_get_chain_kernel(state) -> int:
    k = ctypes.c_int()
    _check(load().ess_get_chain_kernel(state, ctypes.byref(k)))
    return k.value


def ess_set_graphs(state, enable=True):
    _check(load().ess_set_graphs(state, 1 if enable else 0))


def ess_get_tuning(state):
    """(q GEMM tile width, sort_threads) in use (width 0 in the FP64 form)."""
    w, t = ctypes.c_int(), ctypes.c_int()
    _check(load().ess_get_tuning(state, ctypes.byref(w), ctypes.byref(t)))
    return w.value, t.value


def ess_graph_launches(state) -> int:
    n = ctypes.c_longlong()
    _check(load().ess_graph_launches(state, ctypes.byref(n)))
    return n.value


def ess_batch_create(As, bs, cfg: ess_config | None = None):
    """As, bs: sequences of (m_p x d_p) matrices and (m_p,) vectors."""
    d = np.array([np.shape(a)[1] for a in As], dtype=np.int32)
    m = np.array([np.shape(a)[0] for a in As], dtype=np.int32)
    A = _np64(np.concatenate([_np64(a).ravel() for a in As]))
    b = _np64(np.concatenate([_np64(v).ravel() for v in bs]))
    st = _vp()
    _check(load().ess_batch_create(len(As), d.ctypes.data, m.ctypes.data, A.ctypes.data_as(_dp),
                                   b.ctypes.data_as(_dp),
                                   ctypes.byref(cfg) if cfg is not None else None,
                                   ctypes.byref(st)))
    return st


def ess_batch_destroy(batch):
    load().ess_batch_destroy(batch)


def _counts(n_chains):
    return np.ascontiguousarray(n_chains, dtype=np.int32)


def ess_batch_run(batch, n_chains, X, t0, n_iter, seed, samples=None, record_every=0,
                  stream=None):
    nc = _counts(n_chains)
    _check(load().ess_batch_run(batch, nc.ctypes.data, _ptr(X), t0, n_iter, seed, _ptr(samples),
                                record_every, _stream_ptr(stream)))


def ess_batch_step_with_draws(batch, n_chains, X, nu, u, X_next, theta=None, rejected=None,
                              stream=None):
    nc = _counts(n_chains)
    _check(load().ess_batch_step_with_draws(batch, nc.ctypes.data, _ptr(X), _ptr(nu), _ptr(u),
                                            _ptr(X_next), _ptr(theta), _ptr(rejected),
                                            _stream_ptr(stream)))


def ess_batch_products(batch, n_chains, X, nu, P=None, Q=None, stream=None):
    nc = _counts(n_chains)
    _check(load().ess_batch_products(batch, nc.ctypes.data, _ptr(X), _ptr(nu), _ptr(P), _ptr(Q),
                                     _stream_ptr(stream)))


def ess_batch_get_stats(batch) -> dict:
    s = ess_stats()
    _check(load().ess_batch_get_stats(batch, ctypes.byref(s)))
    return s.as_dict()


def ess_batch_reset_stats(batch):
    _check(load().ess_batch_reset_stats(batch))


def ess_batch_set_graphs(batch, enable=True):
    _check(load().ess_batch_set_graphs(batch, 1 if enable else 0))


def ess_batch_set_persistent(batch, enable=True):
    _check(load().ess_batch_set_persistent(batch, 1 if enable else 0))


def ess_batch_selftest_wait(batch, n_chains, X):
    """Bounded dependency-wait self-test of the persistent batched launch (see
    include/ess.h): raises EssError with ESS_ERR_TIMEOUT when the waits gave
    up as they should."""
    nc = _counts(n_chains)
    _check(load().ess_batch_selftest_wait(batch, nc.ctypes.data, _ptr(X)))


def ess_batch_set_timing(batch, enable=True):
    _check(load().ess_batch_set_timing(batch, 1 if enable else 0))


def ess_batch_get_timing(batch) -> dict:
    ms = np.zeros(len(PHASES), dtype=np.float64)
    n = np.zeros(len(PHASES), dtype=np.int64)
    _check(load().ess_batch_get_timing(batch, ms.ctypes.data, n.ctypes.data, len(PHASES)))
    return {p: {"ms": float(ms[i]), "launches": int(n[i])} for i, p in enumerate(PHASES)}


def ess_batch_reset_timing(batch):
    _check(load().ess_batch_reset_timing(batch))


def ess_batch_info(batch) -> dict:
    tx, tp, ni, gl = (ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int(),
                      ctypes.c_longlong())
    _check(load().ess_batch_info(batch, ctypes.byref(tx), ctypes.byref(tp), ctypes.byref(ni),
                                 ctypes.byref(gl)))
    return {"total_x": tx.value, "total_p": tp.value, "n_items": ni.value,
            "graph_launches": gl.value}


def ess_last_error() -> str:
    msg = load().ess_last_error()
    return msg.decode() if msg else ""


# ------------------------------------------------------------ convenience --

class Sampler:
    """Owns an ess_state for D = {x : A x <= b}; X lives in torch CUDA tensors."""

    def __init__(self, A, b, precision=ESS_PREC_FP64, **cfg_overrides):
        cfg = ess_default_config(precision)
        for k, v in cfg_overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.A = _np64(A)
        self.b = _np64(b)
        self.m, self.d = self.A.shape
        self.precision = precision
        self._state = ess_create(self.A, self.b, cfg)

    def close(self):
        if self._state is not None:
            ess_destroy(self._state)
            self._state = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def state(self):
        return self._state

    @property
    def sample_dtype(self):
        import torch
        return torch.float64 if self.precision == ESS_PREC_FP64 else torch.float32

    def run(self, X, n_iter, seed, t0=0, samples=None, record_every=0, stream=None):
        """X: CUDA float64 tensor (n_chains x d), updated in place."""
        n = X.shape[0]
        ess_run(self._state, X, n, t0, n_iter, seed, samples, record_every, stream)
        return X

    def step_with_draws(self, X, nu, u, max_pieces=0, stream=None):
        import torch
        n = X.shape[0]
        dev = X.device
        X_next = torch.empty_like(X)
        theta = torch.empty(n, dtype=torch.float64, device=dev)
        rejected = torch.empty(n, dtype=torch.int32, device=dev)
        n_pieces = torch.empty(n, dtype=torch.int32, device=dev)
        pieces = None
        if max_pieces > 0:
            pieces = torch.zeros((n, max_pieces, 2), dtype=torch.float64, device=dev)
        ess_step_with_draws(self._state, X, nu, u, n, X_next, theta, pieces, max_pieces, n_pieces,
                            rejected, stream)
        return X_next, theta, pieces, n_pieces, rejected

    def products(self, X, nu, stream=None):
        """(A x, A nu) as the state computes them; float64 CUDA tensors."""
        import torch
        n = X.shape[0]
        P = torch.empty((n, self.m), dtype=torch.float64, device=X.device)
        Q = torch.empty((n, self.m), dtype=torch.float64, device=X.device)
        ess_products(self._state, X, nu, n, P, Q, stream)
        return P, Q

    def draw_normals(self, n_chains, t, seed):
        import torch
        out = torch.empty((n_chains, self.d), dtype=self.sample_dtype, device="cuda")
        ess_draw_normals(self._state, n_chains, t, seed, out)
        return out

    def stats(self):
        return ess_get_stats(self._state)

    def reset_stats(self):
        ess_reset_stats(self._state)


class BatchSampler:
    """Owns an ess_batch for the polytopes {x : A_p x <= b_p}; chain states are
    packed problem by problem (chain-major) in one CUDA float64 tensor."""

    def __init__(self, As, bs, precision=ESS_PREC_FP64, **cfg_overrides):
        cfg = ess_default_config(precision)
        for k, v in cfg_overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.As = [_np64(a) for a in As]
        self.bs = [_np64(v) for v in bs]
        self.d = [a.shape[1] for a in self.As]
        self.m = [a.shape[0] for a in self.As]
        self.precision = precision
        self._batch = ess_batch_create(self.As, self.bs, cfg)

    def close(self):
        if self._batch is not None:
            ess_batch_destroy(self._batch)
            self._batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def batch(self):
        return self._batch

    @property
    def sample_dtype(self):
        import torch
        return torch.float64 if self.precision == ESS_PREC_FP64 else torch.float32

    def offsets(self, n_chains):
        """Start of every problem's block in the packed states and products."""
        xo = np.concatenate([[0], np.cumsum([n * d for n, d in zip(n_chains, self.d)])])
        po = np.concatenate([[0], np.cumsum([n * m for n, m in zip(n_chains, self.m)])])
        return xo.astype(np.int64), po.astype(np.int64)

    def pack(self, Xs):
        import torch
        return torch.cat([torch.as_tensor(np.asarray(x, dtype=np.float64)).reshape(-1)
                          for x in Xs]).cuda()

    def unpack(self, flat, n_chains, width="d"):
        w = self.d if width == "d" else self.m
        flat = flat.detach().cpu().numpy() if hasattr(flat, "detach") else np.asarray(flat)
        out, at = [], 0
        for n, k in zip(n_chains, w):
            out.append(flat[at:at + n * k].reshape(n, k))
            at += n * k
        return out

    def run(self, n_chains, X, n_iter, seed, t0=0, samples=None, record_every=0, stream=None):
        ess_batch_run(self._batch, n_chains, X, t0, n_iter, seed, samples, record_every, stream)
        return X

    def step_with_draws(self, n_chains, X, nu, u, stream=None):
        import torch
        n = int(np.sum(n_chains))
        X_next = torch.empty_like(X)
        theta = torch.empty(n, dtype=torch.float64, device=X.device)
        rejected = torch.empty(n, dtype=torch.int32, device=X.device)
        ess_batch_step_with_draws(self._batch, n_chains, X, nu, u, X_next, theta, rejected, stream)
        return X_next, theta, rejected

    def products(self, n_chains, X, nu, stream=None):
        import torch
        tp = int(sum(n * m for n, m in zip(n_chains, self.m)))
        P = torch.empty(tp, dtype=torch.float64, device=X.device)
        Q = torch.empty(tp, dtype=torch.float64, device=X.device)
        ess_batch_products(self._batch, n_chains, X, nu, P, Q, stream)
        return P, Q

    def stats(self):
        return ess_batch_get_stats(self._batch)

    def reset_stats(self):
        ess_batch_reset_stats(self._batch)
