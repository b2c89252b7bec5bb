"""Plain sequential ABC (population Monte Carlo ABC): the weight and proposal
kernels against the float64 oracle, and the final weighted population against
plain prior ABC at the same tolerance."""
import numpy as np
import pytest

from oracle import pmc_oracle as pmc
from tests import inputs
from tests.stats_helpers import assert_posterior_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_14332_gb300 as abc  # noqa: E402
from paper_2012_14332_gb300 import build as _build  # noqa: E402

_build.build()
DEV = torch.device("cuda", 0)
LO = np.zeros(8)
HI = np.array([1, 100, 2, 1, 1, 1, 1, 2.0])


def _population(m, seed):
    g = np.random.default_rng(seed)
    th = (LO + (HI - LO) * (0.3 + 0.4 * g.random((m, 8)))).astype(np.float32)
    w = g.uniform(0.1, 2.0, m)
    return th, w


def test_weights_match_oracle():
    old, w = _population(3000, 1)
    new, _ = _population(5000, 2)
    L = pmc.kernel_factor(old.astype(np.float64), w).astype(np.float32)
    got = abc.abc_pmc_weights(torch.from_numpy(new).to(DEV), torch.from_numpy(old).to(DEV),
                              torch.from_numpy(w).to(DEV), L).cpu().numpy()
    want = pmc.weights(new.astype(np.float64), old.astype(np.float64), w, L.astype(np.float64))
    rel = np.abs(got / want - 1)
    print("pmc weights: median rel %.2e max %.2e" % (np.median(rel), rel.max()))
    assert np.median(rel) < 1e-5 and rel.max() < 1e-3


def test_parents_match_the_oracle_exactly():
    """With a negligible move, each proposal names its parent; the parent index
    (integer work) equals the oracle's inverse-CDF choice from the same Philox
    words: counter (i_lo, i_hi, 0, 4 * 2 + 2), key = seed."""
    import oracle
    m, n, seed, first = 700, 20000, 31, (1 << 32) - 5000
    old, w = _population(m, 6)
    old[:, 0] = 0.25 + 0.5 * np.arange(m) / m              # parent j is read off coordinate 0
    w[::7] = 0.0                                           # zero-weight parents are never chosen
    prop = abc.abc_pmc_propose(torch.from_numpy(old).to(DEV), torch.from_numpy(w).to(DEV),
                               np.eye(8, dtype=np.float32) * 1e-7, n, seed=seed,
                               first_index=first).cpu().numpy().astype(np.float64)
    got = np.rint((prop[:, 0] - 0.25) * m / 0.5).astype(np.int64)
    words = np.array([oracle.philox4x32_10([(first + j) & 0xFFFFFFFF, (first + j) >> 32, 0, 10],
                                           [seed & 0xFFFFFFFF, seed >> 32]) for j in range(n)])
    u = pmc.parent_uniform(words[:, 0], words[:, 1])
    _, want = pmc.propose(old.astype(np.float64), w, np.eye(8) * 1e-7, u, np.zeros((n, 8)), LO, HI)
    assert np.array_equal(got, want)
    assert not np.isin(got, np.arange(0, m, 7)).any()


def test_proposals_have_the_mixture_moments():
    old, w = _population(500, 3)
    L = (pmc.kernel_factor(old.astype(np.float64), w) * 0.01).astype(np.float32)
    n = 1 << 20
    prop = abc.abc_pmc_propose(torch.from_numpy(old).to(DEV), torch.from_numpy(w).to(DEV), L, n, seed=4,
                               first_index=77).cpu().numpy().astype(np.float64)
    assert not np.isnan(prop).any()
    wn = w / w.sum()
    mean = wn @ old.astype(np.float64)
    cov = pmc.weighted_cov(old.astype(np.float64), w) + L.astype(np.float64) @ L.T.astype(np.float64)
    assert np.all(np.abs(prop.mean(0) - mean) < 5 * np.sqrt(np.diag(cov) / n))
    d = np.diag(cov)
    assert np.all(np.abs(np.cov(prop.T) - cov) < 5 * np.sqrt((np.outer(d, d) + cov ** 2) / n))
    # wide moves leave the box: marked NaN in the first coordinate only
    wide = abc.abc_pmc_propose(torch.from_numpy(old).to(DEV), torch.from_numpy(w).to(DEV),
                               np.eye(8, dtype=np.float32) * 50, 4096, seed=5).cpu().numpy()
    out = np.any((wide[:, 1:] < LO[1:]) | (wide[:, 1:] > HI[1:]), axis=1)
    assert np.all(np.isnan(wide[out, 0]))


def test_pmc_posterior_matches_plain_abc():
    w = inputs.workload("region_1e6_T49")
    obs, P = w["observed"], w["P"]
    pilot = abc.abc_distances(obs, P, 1 << 20, 99, mode="fast")
    eps0 = abc.abc_kth_smallest(pilot, 1 << 12)
    info, th, wt, dist = abc.abc_pmc_run(obs, P, eps0, rounds=4, n_particles=4000, batch=1 << 18, max_batches=64,
                                         eps_factor=0.7, seed=8, capacity=1 << 17, mode="fast")
    for r in info:
        print("pmc round eps %.4g sims %d accepted %d ESS %.3f ms %.1f" % (r["eps"], r["n_sims"], r["n_accepted"],
                                                                         r["ess_fraction"], r["ms"]))
    eps_f = info[-1]["eps"]
    assert all(r["n_accepted"] >= 4000 for r in info)
    n_plain = 1 << 26
    th_p, _, _, n_acc_p = abc.abc_sample(obs, P, eps_f, n_plain, 12345, mode="fast", capacity=1 << 18)
    p_prior = n_acc_p / n_plain
    p_pmc = info[-1]["n_accepted"] / info[-1]["n_sims"]
    print("pmc final eps %.4g: prior acceptance %.3e, PMC acceptance %.3e" % (eps_f, p_prior, p_pmc))
    assert p_pmc > 3 * p_prior
    a = th.cpu().numpy().astype(np.float64)
    wa = wt.cpu().numpy()
    b = th_p.cpu().numpy().astype(np.float64)
    assert_posterior_close(a, wa, b, tag="population Monte Carlo")
