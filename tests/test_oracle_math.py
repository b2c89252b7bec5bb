"""Pins of the oracle's exact-mode float32 transcendentals: every coefficient
against a high-precision value of the real number it names, and every function
against float64 libm over (a sweep of) its whole input domain."""
import os
import re

import mpmath as mp
import numpy as np

import oracle

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "abc_oracle.c")


def _rn32(x):
    """Correctly rounded float32 of an mpmath real."""
    f = np.float32(float(x))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    return min(cands, key=lambda c: abs(mp.mpf(float(c)) - x))


def test_coefficients_are_correctly_rounded_values():
    mp.mp.prec = 200
    ln2 = mp.log(2)
    want = {
        "LN2_F": ln2, "NEG_2LN2_F": -2 * ln2, "PI_F": mp.pi, "SQRT2_F": mp.sqrt(2),
        "LOG_C1": 2 / (1 * ln2), "LOG_C3": 2 / (3 * ln2), "LOG_C5": 2 / (5 * ln2),
        "LOG_C7": 2 / (7 * ln2), "LOG_C9": 2 / (9 * ln2),
        "SIN_C3": -1 / mp.factorial(3), "SIN_C5": 1 / mp.factorial(5), "SIN_C7": -1 / mp.factorial(7),
        "SIN_C9": 1 / mp.factorial(9),
        "COS_C2": -1 / mp.factorial(2), "COS_C4": 1 / mp.factorial(4), "COS_C6": -1 / mp.factorial(6),
        "COS_C8": 1 / mp.factorial(8), "COS_C10": -1 / mp.factorial(10),
    }
    for j in range(2, 8):
        want["EXP_C%d" % j] = 1 / mp.factorial(j)
    src = open(SRC).read()
    found = dict(re.findall(r"static const float (\w+) = (-?0x[0-9a-fA-F.]+p[-+]?\d+)f;", src))
    assert set(want) == set(found), set(want) ^ set(found)
    for name, real in want.items():
        assert np.float32(float.fromhex(found[name])) == _rn32(mp.mpf(real)), name


def _ulp_err(got, ref):
    got = got.astype(np.float64)
    ulp = np.spacing(np.abs(got.astype(np.float32))).astype(np.float64)
    return np.abs(got - ref) / ulp


def test_log2x_on_every_uniform_lattice_point():
    """log2 of every u = (2m+1) 2^-24 (all 2^23 Box-Muller inputs): <= 3 ulp."""
    m = np.arange(0, 1 << 23, dtype=np.float64)
    u = ((2 * m + 1) * 2.0**-24).astype(np.float32)
    y = oracle.log2x_batch(u)
    ref = np.log2(u.astype(np.float64))
    assert np.max(_ulp_err(y, ref)) <= 3.0


def test_log2x_on_counts():
    """log2 of integer counts 1 .. 2^31 (the pow in Eq. 4): <= 1 ulp; exact on powers of two."""
    x = np.unique(np.concatenate([np.arange(1, 1 << 20), np.geomspace(1, 2**31, 1 << 20).astype(np.int64)]))
    xf = x.astype(np.float32)
    y = oracle.log2x_batch(xf)
    ref = np.log2(xf.astype(np.float64))
    nz = ref != 0
    assert np.max(_ulp_err(y[nz], ref[nz])) <= 1.0
    assert y[x == 1][0] == 0.0
    p2 = 2.0 ** np.arange(0, 31)
    assert np.array_equal(oracle.log2x_batch(p2.astype(np.float32)), np.arange(0, 31).astype(np.float32))


def test_exp2x_bound_and_edges():
    y = np.concatenate([np.linspace(-125, 127, 1 << 21), np.linspace(-1, 1, 1 << 18)]).astype(np.float32)
    e = oracle.exp2x_batch(y)
    ref = np.exp2(y.astype(np.float64))
    assert np.max(_ulp_err(e, ref)) <= 1.5
    k = np.arange(-125, 128).astype(np.float32)
    assert np.array_equal(oracle.exp2x_batch(k), np.exp2(k.astype(np.float64)).astype(np.float32))
    assert oracle.exp2x(127.5) == np.inf and oracle.exp2x(1e30) == np.inf
    assert oracle.exp2x(-125.6) == 0.0
    assert oracle.exp2x(0.0) == 1.0


def test_sincospix_on_every_angle_lattice_point():
    """sin / cos(pi v) for every v = 2u (all 2^23 Box-Muller angles): abs err <= 1e-7."""
    m = np.arange(0, 1 << 23, dtype=np.float64)
    v = (2 * (2 * m + 1) * 2.0**-24).astype(np.float32)
    s, c = oracle.sincospix_batch(v)
    vd = v.astype(np.float64)
    assert np.max(np.abs(s - np.sin(np.pi * vd))) <= 1e-7
    assert np.max(np.abs(c - np.cos(np.pi * vd))) <= 1e-7
    # exact at the quarter turns
    for vv, (ss, cc) in {0.0: (0, 1), 0.5: (1, 0), 1.0: (0, -1), 1.5: (-1, 0), 2.0: (0, 1)}.items():
        a, b = oracle.sincospix(vv)
        assert a == ss and b == cc
    # odd/even symmetry on a sweep
    w = np.linspace(-0.999, 0.999, 4097).astype(np.float32)
    s1, c1 = oracle.sincospix_batch(w)
    s2, c2 = oracle.sincospix_batch(-w)
    assert np.array_equal(s1, -s2) and np.array_equal(c1, c2)
