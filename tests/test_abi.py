"""The C-ABI library builds, loads and exports every symbol include/ess.h declares.

CPU-only: no GPU compute call is made.  The host-side whitening helpers
(App. A) are checked against the oracle.
"""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2407_10449_gb300 as ess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ess.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ess_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_binding_names():
    assert _declared() == sorted(ess.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = ess.load()
    out = subprocess.run(["nm", "-D", "--defined-only", ess.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_default_config():
    c64 = ess.ess_default_config(ess.ESS_PREC_FP64)
    cmx = ess.ess_default_config(ess.ESS_PREC_MIXED)
    assert c64.refresh_k == 32 and cmx.refresh_k == 32
    assert c64.tangent_thresh == pytest.approx(1e-4)
    assert c64.trim_eps == 0.0
    assert cmx.precision == ess.ESS_PREC_MIXED
    with pytest.raises(ess.EssError):
        ess.ess_default_config(7)


def test_whiten_matches_oracle():
    rng = np.random.default_rng(0)
    d, m = 7, 11
    A = rng.standard_normal((m, d))
    b = rng.uniform(0.1, 1.0, m)
    mu = rng.standard_normal(d)
    M = rng.standard_normal((d, d))
    L = np.linalg.cholesky(M @ M.T + np.eye(d))
    Aw, bw = ess.ess_whiten(A, b, mu, L)
    Ao, bo = oracle.whiten(A, b, mu, L)
    np.testing.assert_allclose(Aw, Ao, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(bw, bo, rtol=1e-13, atol=1e-14)
    U = rng.standard_normal((5, d))
    np.testing.assert_allclose(ess.ess_unwhiten(L, mu, U), oracle.unwhiten(L, mu, U),
                               rtol=1e-13, atol=1e-14)
    # mu = NULL means zero
    Aw0, bw0 = ess.ess_whiten(A, b, None, L)
    np.testing.assert_allclose(bw0, b)


def test_argument_errors_without_gpu():
    with pytest.raises(ess.EssError) as e:
        ess.ess_whiten(np.zeros((0, 3)), np.zeros(0), None, np.eye(3))
    assert e.value.status == ess.ESS_ERR_ARG


def test_float_scaling_range_is_checked_without_gpu():
    """The mixed form (A, b, p, q in float; b^2 against p^2 + q^2) refuses
    rows whose largest entry lies outside [2^-30, 2^30] and b beyond 2^30;
    the FP64 form's split products (row scales kept as floats) refuse rows
    outside [2^-100, 2^100].  Both before touching the GPU; the batched
    mixed form likewise."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 4))
    b = np.ones(6)
    cases = []
    for scale in (1e40, 1e-41):
        A2 = A.copy()
        A2[2] *= scale
        cases += [(A2, b, dict(precision=ess.ESS_PREC_MIXED)),
                  (A2, b, dict(precision=ess.ESS_PREC_FP64,
                               fp64_products=ess.ESS_PRODUCTS_SPLIT))]
    b2 = b.copy()
    b2[4] = 1e10
    cases.append((A, b2, dict(precision=ess.ESS_PREC_MIXED)))
    A4 = A.copy()
    A4[0] *= 1e12  # inside the split products' range, outside the mixed form's
    cases.append((A4, b, dict(precision=ess.ESS_PREC_MIXED)))
    for Ax, bx, cfg in cases:
        with pytest.raises(ess.EssError) as e:
            ess.Sampler(Ax, bx, **cfg)
        assert e.value.status == ess.ESS_ERR_ARG
        assert "scaling range" in str(e.value)
    A3 = A.copy()
    A3[1] *= 1e40
    with pytest.raises(ess.EssError) as e:
        ess.BatchSampler([A, A3], [b, b], precision=ess.ESS_PREC_MIXED)
    assert e.value.status == ess.ESS_ERR_ARG

