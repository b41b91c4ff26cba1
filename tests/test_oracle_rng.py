"""Pins for the oracle's counter-based RNG: Philox4x32-10 (Salmon et al., SC'11)
and the Box-Muller normals that drive xi in the PnP-ULA update (Eq. 8).

Pins: an independent library implementation of Philox4x32-10 (Triton's,
executed by its CPU interpreter); the Box-Muller identities that fix which
uniform feeds the radius and which the angle; moments and a KS test of the
normals; independence of the (t, chain) streams.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

_TRITON_SCRIPT = textwrap.dedent(r"""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl

    @triton.jit
    def k(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m).to(tl.uint32)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m).to(tl.uint32)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m).to(tl.uint32)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m).to(tl.uint32)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a.to(tl.int64) & 0xffffffff, mask=m)
        tl.store(out_ptr + 4 * i + 1, b.to(tl.int64) & 0xffffffff, mask=m)
        tl.store(out_ptr + 4 * i + 2, c.to(tl.int64) & 0xffffffff, mask=m)
        tl.store(out_ptr + 4 * i + 3, d.to(tl.int64) & 0xffffffff, mask=m)

    req = json.loads(sys.stdin.read())
    res = []
    for seed, ctrs in req:
        c = torch.tensor(ctrs, dtype=torch.int64).reshape(-1)
        out = torch.zeros_like(c)
        k[(1,)](out, c, seed, len(ctrs), BLOCK=64)
        res.append(out.reshape(-1, 4).tolist())
    print(json.dumps(res))
""")


def _triton_philox(cases):
    import json
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES=""))
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_philox_matches_library_implementation(orc):
    rng = np.random.default_rng(1)
    seeds = [0, 1, 0x1234_5678_9ABC_DEF0, 2 ** 64 - 1, 1100]
    cases = []
    for s in seeds:
        ctrs = rng.integers(0, 2 ** 32, size=(40, 4), dtype=np.uint64)
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [2 ** 32 - 1] * 4
        ctrs[2] = [5, 17, 3, 0]          # layout used by the sampler: (n/4, t, chain, 0)
        cases.append([s if s < 2 ** 63 else s - 2 ** 64, ctrs.astype(np.int64).tolist()])
    ref = _triton_philox(cases)
    for (s, ctrs), r in zip(cases, ref):
        s = s % 2 ** 64
        key = np.array([s & 0xFFFFFFFF, s >> 32], dtype=np.uint32)
        got = orc.philox4x32_10(np.array(ctrs, dtype=np.uint64).astype(np.uint32), key)
        np.testing.assert_array_equal(got.astype(np.int64), np.array(r, dtype=np.int64))


def test_box_muller_pairing(orc):
    """xi[4m]^2 + xi[4m+1]^2 = -2 ln u0 and atan2(xi[4m+1], xi[4m]) = 2 pi u1 (mod 2 pi),
    with u_k = ((word_k >> 8) + 1/2) 2^-24 of Philox((m, t, chain, 0), seed)."""
    seed, t, chain = 0xDEADBEEF01, 7, 3
    n = 64
    xi = orc.normals(seed, t, chain, n)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    ctr = np.array([[m, t, chain, 0] for m in range(n // 4)], dtype=np.uint32)
    words = orc.philox4x32_10(ctr, key)
    u = ((words >> 8).astype(np.float64) + 0.5) / 2 ** 24
    for pair in range(2):
        r2 = xi[2 * pair::4] ** 2 + xi[2 * pair + 1::4] ** 2
        np.testing.assert_allclose(r2, -2 * np.log(u[:, 2 * pair]), rtol=1e-12)
        ang = np.mod(np.arctan2(xi[2 * pair + 1::4], xi[2 * pair::4]), 2 * np.pi)
        np.testing.assert_allclose(ang, 2 * np.pi * u[:, 2 * pair + 1], rtol=0, atol=1e-9)


def test_normals_are_standard_normal(orc):
    xi = orc.normals(12345, 0, 0, 200_000)
    assert abs(xi.mean()) < 5 / np.sqrt(xi.size)
    assert abs(xi.var() - 1) < 5 * np.sqrt(2 / xi.size)
    assert stats.kstest(xi, "norm").pvalue > 1e-4


def test_streams_are_independent(orc):
    a = orc.normals(99, 0, 0, 100_000)
    b = orc.normals(99, 1, 0, 100_000)
    c = orc.normals(99, 0, 1, 100_000)
    d = orc.normals(100, 0, 0, 100_000)
    for u, v in ((a, b), (a, c), (a, d), (b, c)):
        assert abs(np.corrcoef(u, v)[0, 1]) < 5 / np.sqrt(u.size)


def test_normals_prefix_consistency(orc):
    """The draw for pixel n depends only on (seed, t, chain, n): a shorter request is a prefix."""
    a = orc.normals(5, 2, 1, 1001)
    b = orc.normals(5, 2, 1, 37)
    np.testing.assert_array_equal(a[:37], b)
