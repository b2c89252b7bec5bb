"""Pins of the population Monte Carlo ABC oracle: the weights against SciPy's
multivariate normal density, the proposal distribution's mean and covariance
against the closed form (weighted mean; weighted covariance plus Sigma), and
the kernel variance 2 Cov_w."""
import numpy as np
from scipy import stats

from oracle import pmc_oracle as pmc

LO = np.zeros(8)
HI = np.array([1, 100, 2, 1, 1, 1, 1, 2.0])


def _particles(n, seed):
    g = np.random.default_rng(seed)
    th = LO + (HI - LO) * (0.3 + 0.4 * g.random((n, 8)))
    w = g.uniform(0.1, 2.0, n)
    return th, w


def test_weights_match_multivariate_normal_density():
    old, w = _particles(300, 1)
    new, _ = _particles(50, 2)
    L = pmc.kernel_factor(old, w)
    S = L @ L.T
    assert np.allclose(S, 2 * pmc.weighted_cov(old, w))
    got = pmc.weights(new, old, w, L)
    norm = np.sqrt((2 * np.pi) ** 8 * np.linalg.det(S))
    dens = np.array([sum(w[j] * stats.multivariate_normal(old[j], S).pdf(x) for j in range(len(old))) for x in new])
    assert np.allclose(1.0 / got, dens * norm, rtol=1e-8)


def test_proposals_have_the_mixture_moments():
    old, w = _particles(200, 3)
    L = pmc.kernel_factor(old, w) * 0.01      # keep proposals inside the box
    g = np.random.default_rng(4)
    n = 200_000
    prop, parents = pmc.propose(old, w, L, g.random(n), g.normal(size=(n, 8)), LO, HI)
    assert not np.isnan(prop).any()
    wn = w / w.sum()
    mean = wn @ old
    cov = pmc.weighted_cov(old, w) + L @ L.T
    se = np.sqrt(np.diag(cov) / n)
    assert np.all(np.abs(prop.mean(0) - mean) < 5 * se)
    d = np.diag(cov)
    se_c = np.sqrt((np.outer(d, d) + cov ** 2) / n)         # standard error of a sample covariance
    assert np.all(np.abs(np.cov(prop.T) - cov) < 5 * se_c)
    # parents are drawn with probability w / sum w
    freq = np.bincount(parents, minlength=len(w)) / n
    assert np.all(np.abs(freq - wn) < 5 * np.sqrt(wn * (1 - wn) / n) + 1e-9)


def test_proposals_outside_the_box_are_marked():
    old, w = _particles(20, 5)
    L = np.eye(8) * 100.0
    prop, _ = pmc.propose(old, w, L, np.linspace(0, 0.99, 50), np.ones((50, 8)), LO, HI)
    assert np.all(np.isnan(prop[:, 0]))


def test_parent_uniform_spans_the_unit_interval():
    """The 53-bit construction: zero words give 0, all-ones words give the
    largest double below 1, and each bit of the kept fields lands at its own
    power of two (so no field is dropped or overlapped)."""
    assert pmc.parent_uniform(0, 0) == 0.0
    assert pmc.parent_uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert pmc.parent_uniform(0x80000000, 0) == 0.5
    assert pmc.parent_uniform(0x20, 0) == 2.0 ** -27
    assert pmc.parent_uniform(0, 0x40) == 2.0 ** -53
    assert pmc.parent_uniform(0x1F, 0x3F) == 0.0                 # the dropped low bits
    w = np.random.default_rng(0).integers(0, 1 << 32, size=(2, 200000), dtype=np.uint64)
    u = pmc.parent_uniform(w[0], w[1])
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / len(u))
    assert u.min() >= 0 and u.max() < 1


def test_parent_choice_is_the_inverse_cdf():
    """Parents from evenly spaced uniforms land in proportion to the weights."""
    w = np.array([1.0, 3.0, 0.0, 4.0])
    u = (np.arange(8000) + 0.5) / 8000
    _, j = pmc.propose(np.zeros((4, 8)), w, np.eye(8) * 1e-9, u, np.zeros((8000, 8)), -np.ones(8), np.ones(8))
    assert np.array_equal(np.bincount(j, minlength=4), [1000, 3000, 0, 4000])
