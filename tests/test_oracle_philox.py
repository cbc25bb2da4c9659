"""Pins of the oracle's Philox4x32-10 and of its draw mapping.

The generator is pinned to an implementation the oracle does not share:
triton's Philox4x32-10 (the 32-bit branch of ``triton.language.philox``), run
on the CPU through triton's interpreter in a child process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def k(out_ptr, c_ptr, seed, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    n = len(ctrs)
    flat = [v - (1 << 32) if v >= (1 << 31) else v for c in ctrs for v in c]
    ctr = torch.tensor(flat, dtype=torch.int32)
    out = torch.zeros(4 * n, dtype=torch.int32)
    k[(1,)](out, ctr, seed, N=n)
    res.append([v & 0xFFFFFFFF for v in out.tolist()])
print(json.dumps(res))
"""


def test_philox_matches_triton(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(12345)
    cases = []
    for seed in [0, 1, 7, 11, 0x123456789, 0xFFFFFFFFFFFFFFFF, 2**32, 1000 + 4095]:
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).tolist()
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [0xFFFFFFFF] * 4
        cases.append([seed, ctrs])
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, "-c", TRITON_SCRIPT], input=json.dumps(cases),
                          capture_output=True, text=True, env=env, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for (seed, ctrs), want in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i, c in enumerate(ctrs):
            got = orc.philox4x32_10(c, key).tolist()
            assert got == want[4 * i:4 * i + 4], (seed, c)


def test_philox_bits_are_balanced(orc):
    # 4096 blocks = 2^19 bits; the number of ones is Binomial(n, 1/2).
    ones = 0
    n = 0
    for g in range(4096):
        w = orc.philox4x32_10([g, 0, 3, 0], [7, 0])
        ones += sum(bin(int(v)).count("1") for v in w)
        n += 128
    z = (ones - n / 2) / np.sqrt(n / 4)
    assert abs(z) < 5


def test_site_uniform_mapping(orc):
    """The k-bit draw of a site is read MSB first from words (g, j) at bit b,
    with g = i // 128, j = (i % 128) // 32, b = i % 32, i = y*L + x."""
    seed, L, t = 0xABCDEF0123, 96, 5
    for (x, y) in [(0, 0), (31, 0), (32, 0), (95, 0), (0, 1), (40, 7), (95, 95)]:
        i = y * L + x
        g, j, b = i // 128, (i % 128) // 32, i % 32
        for k in (1, 3, 32):
            U = 0
            for m in range(k):
                w = orc.philox4x32_10([g & 0xFFFFFFFF, g >> 32, t, m],
                                      [seed & 0xFFFFFFFF, seed >> 32])
                U = (U << 1) | ((int(w[j]) >> b) & 1)
            assert orc.site_uniform(seed, L, x, y, t, k) == U


def test_site_uniform_is_uniform(orc):
    # chi-square of 3-bit draws over 4096 sites against the uniform law on [0, 8)
    from scipy import stats
    L = 64
    counts = np.zeros(8)
    for i in range(4096):
        counts[orc.site_uniform(99, L, i % L, i // L, 17, 3)] += 1
    assert stats.chisquare(counts).pvalue > 1e-3
