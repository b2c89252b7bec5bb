"""The statistics the GPU tests of the sequential samplers rely on, checked by
simulation where the answer is known: under a true null (an importance-
weighted sample and a plain sample of one distribution) the sandwich-variance
z-scores are calibrated even when the weights pile up in one tail, and they
detect a small shift; the n_eff-scaled Kolmogorov test is shown to over-reject
with such weights (why it is not used there)."""
import numpy as np
from scipy import stats

from tests.stats_helpers import cdf_z_scores, sandwich_ks, weighted_ks, weighted_mean_z


def _draw(rng, n, mu, sd, shift):
    x = rng.normal(mu, sd, n)
    w = stats.norm.pdf(x) / stats.norm.pdf(x, mu, sd)
    y = rng.normal(shift, 1.0, n)
    return x, w, y


def test_unweighted_case_reduces_to_the_plain_statistics():
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=3000), rng.normal(size=3000)
    D, p, ne = sandwich_ks(x, np.ones(3000), y)
    ks = stats.ks_2samp(x, y)
    assert abs(D - ks.statistic) < 1e-12 and abs(ne - 3000) < 1e-6
    assert abs(p - weighted_ks(x, np.ones(3000), y)[1]) < 1e-12
    z = weighted_mean_z(x, np.ones(3000), y)
    assert abs(z - (x.mean() - y.mean()) / np.sqrt(x.var() / 3000 + y.var() / 3000)) < 1e-9


def test_sandwich_z_scores_are_calibrated_with_tail_heavy_weights():
    rng = np.random.default_rng(1)
    zc, zm, pk = [], [], []
    for _ in range(150):
        x, w, y = _draw(rng, 10000, 0.5, 0.7, 0.0)   # a narrow, shifted proposal: ESS about 23 %
        zc.append(np.abs(cdf_z_scores(x, w, y)).max())
        zm.append(abs(weighted_mean_z(x, w, y)))
        pk.append(weighted_ks(x, w, y)[1])
    zc, zm, pk = np.array(zc), np.array(zm), np.array(pk)
    assert (zc > 4).mean() <= 0.02 and (zm > 4).mean() <= 0.02
    # the n_eff-scaled KS rejects the true null far above its nominal 1 %
    assert (pk < 0.01).mean() > 0.05


def test_sandwich_z_scores_detect_a_small_shift():
    rng = np.random.default_rng(2)
    hits = [np.abs(cdf_z_scores(*_draw(rng, 20000, 0.5, 0.7, 0.1))).max() > 4 for _ in range(40)]
    assert np.mean(hits) > 0.75


def test_posterior_error_measures_a_known_shift():
    """A plain sample against itself shifted by 0.1 sd: the mean error reads
    0.1 sd and the CDF error about phi(0) 0.1; the accuracy check rejects a
    0.1 sd shift and accepts 0.02 sd at these sizes."""
    from tests.stats_helpers import assert_posterior_close, posterior_error
    rng = np.random.default_rng(3)
    y = rng.normal(size=(200000, 1))
    x = rng.normal(size=(200000, 1))
    dm, se_m, dc, se_c = posterior_error(x[:, 0] + 0.1, np.ones(len(x)), y[:, 0])
    assert abs(dm - 0.1) < 5 * se_m and abs(dc - 0.1 * stats.norm.pdf(0)) < 0.01
    import pytest
    with pytest.raises(AssertionError):
        assert_posterior_close(x + 0.1, np.ones(len(x)), y)
    assert_posterior_close(x + 0.02, np.ones(len(x)), y)
