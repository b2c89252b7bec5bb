"""Pins of the oracle's random-number layer (Philox4x32-10, uniforms, prior
draw, Box-Muller normals) against things other than itself: a third-party
Philox implementation, closed-form moments and exact lattice structure."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

import oracle
from tests import inputs

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def _k(out, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i), 10)
    tl.store(out + i * 4 + 0, a)
    tl.store(out + i * 4 + 1, b)
    tl.store(out + i * 4 + 2, c)
    tl.store(out + i * 4 + 3, d)

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    c = torch.tensor(ctrs, dtype=torch.int64).to(torch.uint32)
    N = c.shape[0]
    out = torch.zeros(4 * N, dtype=torch.uint32)
    cols = [c[:, j].contiguous() for j in range(4)]
    _k[(1,)](out, cols[0], cols[1], cols[2], cols[3], seed, N=N)
    res.append([int(x) & 0xFFFFFFFF for x in out.tolist()])
print(json.dumps(res))
"""


def test_philox_matches_triton_interpreter():
    """Philox4x32-10 against Triton's own implementation (run on the CPU by
    Triton's interpreter): an independent third-party code of the same
    published generator (Salmon et al., SC'11)."""
    pytest.importorskip("triton")
    g = inputs.rng(11)
    req = []
    seeds = [0, 1, 0xFFFFFFFF, 0x123456789ABCDEF0, 20201228, 1234]
    for s in seeds:
        ctrs = g.integers(0, 2**32, size=(16, 4), dtype=np.uint64)
        ctrs[0] = 0
        ctrs[1] = 0xFFFFFFFF
        req.append([s, ctrs.tolist()])
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req), capture_output=True,
                       text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    res = json.loads(p.stdout.strip().splitlines()[-1])
    for (s, ctrs), got in zip(req, res):
        key = [s & 0xFFFFFFFF, (s >> 32) & 0xFFFFFFFF]
        for j, c in enumerate(ctrs):
            ours = oracle.philox4x32_10(c, key)
            assert list(map(int, ours)) == got[4 * j:4 * j + 4], (s, c)


def test_philox_zero_vector_and_avalanche():
    # all-zero counter and key: a fixed known output of the generator
    out = oracle.philox4x32_10([0, 0, 0, 0], [0, 0])
    assert [int(x) for x in out] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    # flipping one input bit flips about half of the 128 output bits
    g = inputs.rng(3)
    flips = []
    for _ in range(200):
        c = g.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        k = g.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
        b = int(g.integers(0, 4))
        c2 = c.copy()
        c2[b] ^= np.uint32(1 << int(g.integers(0, 32)))
        o1, o2 = oracle.philox4x32_10(c, k), oracle.philox4x32_10(c2, k)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(o1, o2)))
    assert abs(np.mean(flips) - 64) < 2.0


def test_uniform_is_odd_lattice():
    """u = (2m+1) 2^-24 with m = w mod 2^23: exact, in (0, 1)."""
    g = inputs.rng(5)
    w = g.integers(0, 2**32, size=1 << 16, dtype=np.uint64).astype(np.uint32)
    w = np.concatenate([w, np.array([0, 0x7FFFFF, 0x800000, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)])
    u = oracle.uniform_batch(w).astype(np.float64)
    m = (w & 0x7FFFFF).astype(np.float64)
    assert np.array_equal(u * 2.0**24, 2 * m + 1)
    assert u.min() > 0 and u.max() < 1
    assert oracle.uniform(0) == np.float32(2.0**-24)
    assert oracle.uniform(0xFFFFFFFF) == np.float32(1 - 2.0**-24)


def test_prior_draw_moments_and_support():
    """theta_j ~ U(lo_j, hi_j) (Sec. 2.1, Eq. 2): support, mean, variance."""
    n = 1 << 17
    th = oracle.prior_batch(1234, 0, 0, n).astype(np.float64)
    lo, hi = inputs.PAPER_LO.astype(np.float64), inputs.PAPER_HI.astype(np.float64)
    assert np.all(th >= lo) and np.all(th <= hi)
    assert np.all(th > 0)
    mean = th.mean(axis=0)
    var = th.var(axis=0)
    sd_mean = (hi - lo) / np.sqrt(12 * n)
    assert np.all(np.abs(mean - (lo + hi) / 2) < 5 * sd_mean)
    # var of a uniform sample variance: (hi-lo)^4 (1/80 - 1/144) / n
    sd_var = (hi - lo) ** 2 * np.sqrt((1 / 80 - 1 / 144) / n)
    assert np.all(np.abs(var - (hi - lo) ** 2 / 12) < 5 * sd_var)
    # coordinates are uncorrelated
    c = np.corrcoef(th.T)
    assert np.all(np.abs(c - np.eye(8)) < 5 / np.sqrt(n))


def test_prior_draw_degenerate_box_and_streams():
    lo = np.array([0.3, 7, 1.5, 0.2, 0.1, 0.05, 0.5, 1.0], dtype=np.float32)
    th = oracle.prior_draw(99, 0, 17, lo=lo, hi=lo)
    assert np.array_equal(th, lo)
    a = oracle.prior_draw(99, 0, 17)
    assert not np.array_equal(a, oracle.prior_draw(99, 1, 17))
    assert not np.array_equal(a, oracle.prior_draw(98, 0, 17))
    assert not np.array_equal(a, oracle.prior_draw(99, 0, 18))
    assert not np.array_equal(a, oracle.prior_draw(99, 0, 17 + (1 << 32)))


def test_box_muller_normals_moments_ks():
    """Normals of the day-pair blocks: N(0,1) moments, KS against Phi,
    independence within a pair, and the truncation |z| <= sqrt(-2 ln 2^-24)."""
    n = 1 << 16
    z = oracle.normals_batch(20201228, 0, 0, n, 1).astype(np.float64)
    flat = z.ravel()
    N = flat.size
    assert abs(flat.mean()) < 5 / np.sqrt(N)
    assert abs(flat.var() - 1) < 5 * np.sqrt(2 / N)
    assert abs(stats.skew(flat)) < 5 * np.sqrt(6 / N)
    assert abs(stats.kurtosis(flat, fisher=False) - 3) < 5 * np.sqrt(24 / N)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    for p in range(5):
        r = np.corrcoef(z[:, 2 * p], z[:, 2 * p + 1])[0, 1]
        assert abs(r) < 5 / np.sqrt(n)
    assert np.abs(flat).max() <= np.sqrt(-2 * np.log(2.0**-24)) + 1e-5
    # different day pairs give different normals
    z2 = oracle.normals_batch(20201228, 0, 0, 16, 2)
    assert not np.array_equal(z2, z[:16].astype(np.float32))


def test_box_muller_against_float64_formula():
    """z = sqrt(-2 ln u1) (cos, sin)(2 pi u2) within the exact-mode error
    bound (log2 <= 3 ulp, sinpi/cospi <= 1e-7 abs, two roundings)."""
    g = inputs.rng(9)
    w = g.integers(0, 2**32, size=(4096, 2), dtype=np.uint64).astype(np.uint32)
    for a, b in w:
        z = oracle.box_muller(int(a), int(b)).astype(np.float64)
        u1 = (2 * (int(a) & 0x7FFFFF) + 1) * 2.0**-24
        u2 = (2 * (int(b) & 0x7FFFFF) + 1) * 2.0**-24
        r = np.sqrt(-2 * np.log(u1))
        ref = np.array([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        assert np.all(np.abs(z - ref) <= 4e-7 * (1 + r)), (a, b, z, ref)
