"""Pin of the oracle's Philox4x32-10 bit stream against an independent
implementation: the Philox generator of triton's language library (written by
other authors from Salmon et al. 2011, with the published round multipliers
and Weyl key increments), run on the host by triton's interpreter.

The oracle's block function (oracle.philox4x32_10: 4-word counter, 2-word
key, ten rounds) must give the library's four output words bit for bit on
random counters and keys and on the edge words (0 and 2^32 - 1), which pins
the multipliers, the key schedule, the carries of the 32 x 32 -> 64 products
and the output word order.  The CUDA draws equal the oracle's blocks bit for
bit (tests/test_gpu_run.py), so this pins them as well.  The library maps a
64-bit seed s to the key (s mod 2^32, s div 2^32).

The interpreter runs in a child process (it is switched on by an environment
variable read when triton is imported); without triton the test is skipped.
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

CHILD = textwrap.dedent("""
    import json, sys
    import numpy as np
    import torch
    import triton
    import triton.language as tl

    @triton.jit
    def blocks(c_ptr, out_ptr, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c_ptr + 4 * i)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        o0, o1, o2, o3 = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i, o0)
        tl.store(out_ptr + 4 * i + 1, o1)
        tl.store(out_ptr + 4 * i + 2, o2)
        tl.store(out_ptr + 4 * i + 3, o3)

    req = json.load(sys.stdin)
    res = []
    for seed, ctrs in req:
        ctr = np.array(ctrs, dtype=np.uint32)
        c = torch.from_numpy(ctr.view(np.int32).copy())
        out = torch.zeros_like(c)
        blocks[(1,)](c, out, seed, N=ctr.shape[0])
        res.append(out.numpy().view(np.uint32).tolist())
    json.dump(res, sys.stdout)
""")


def _library_blocks(req):
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", CHILD], input=json.dumps(req), env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.fail("triton interpreter run failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout)


def test_philox_matches_an_independent_library_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(2011)
    edge = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF]
    seeds = [0, 1, 0xFFFFFFFF, 0x100000000, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF] + [
        int(s) for s in rng.integers(0, 2**63, size=4)]
    req = []
    for seed in seeds:
        ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
        for j, e in enumerate(edge):  # edge words in every position
            ctr[4 * j:4 * j + 4] = e
            ctr[4 * j + 1, j % 4] = edge[(j + 2) % len(edge)]
        req.append([seed, ctr.tolist()])
    got = _library_blocks(req)
    n = 0
    for (seed, ctrs), lib in zip(req, got):
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        for ctr, want in zip(ctrs, lib):
            ours = oracle.philox4x32_10(np.array(ctr, dtype=np.uint32), key)
            assert list(map(int, ours)) == want, (hex(seed), ctr)
            n += 1
    assert n == len(seeds) * 64
