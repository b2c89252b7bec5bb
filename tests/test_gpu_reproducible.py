"""Reproducible learned proposals: a seed fixes the trained flows.

The flow gradient takes no float atomics (the tensor-memory accumulations run
in a fixed job order, the CTAs' partials are added in a fixed tree), and the
sequential drivers put each run's accepted samples in sample-index order
before weighting, pooling and training. So a gradient computed twice is the
same bit for bit, in both CTA forms, and two sequential-ABC runs with one seed
give the same rounds, accepted samples, weights and distances bit for bit;
another seed gives other ones. Population Monte Carlo ABC keeps each round's
population in sample-index order, with the same consequence."""
import numpy as np
import pytest

from tests import inputs

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


def _thetas(n, seed):
    u = np.random.default_rng(seed).uniform(0.02, 0.98, size=(n, 8))
    return torch.from_numpy((LO + (HI - LO) * u).astype(np.float32)).to(DEV)


@pytest.mark.parametrize("n_flows,n", [(1, 5000), (1, 1 << 16), (16, 2055)])
def test_gradient_is_the_same_on_every_call(n_flows, n):
    """One flow over 5,000 and 65,536 rows (4-warp CTAs, paired at 256 hidden
    units; the second fills every SM) and a set of 16 flows (15-warp CTAs):
    three calls, one result."""
    f = abc.Flow(3, 256, n_flows=n_flows)
    f.init_random(seed=3, scale=0.5)
    th = _thetas(n, 11)
    w = torch.from_numpy(np.random.default_rng(12).uniform(0.2, 2.0, size=n).astype(np.float32)).to(DEV)
    loss0, g0 = f.gradient(th, w)
    for _ in range(2):
        loss, g = f.gradient(th, w)
        assert loss == loss0 and np.array_equal(g, g0)
    assert np.count_nonzero(g0) > 0.3 * g0.size
    f.close()


def _no_times(rounds):
    """Round records without their stage timings (which vary from run to run)."""
    if rounds and isinstance(rounds[0], list):
        return [_no_times(r) for r in rounds]
    return [{k: v for k, v in r.items() if not k.startswith("ms_")} for r in rounds]


def _smc(seed):
    w = inputs.workload("region_1e6_T49")
    obs, P = w["observed"], w["P"]
    eps0 = 2.2 * w["eps"]
    info, th, wt, dist = abc.abc_smc_run(obs, P, eps0, rounds=3, sims_per_round=1 << 18, eps_factor=0.7,
                                         flow_blocks=3, flow_hidden=128, train_steps=150, train_batch=1024,
                                         train_lr=2e-3, seed=seed, mode="fast")
    return _no_times(info), th.cpu().numpy(), wt.cpu().numpy(), dist.cpu().numpy()


def test_sequential_abc_is_the_same_for_one_seed():
    a, b, c = _smc(5), _smc(5), _smc(6)
    assert [r["proposal"] for r in a[0]][-1] == 1, "the last round should draw from the trained flow"
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    assert a[1].shape[0] > 100
    assert a[0] != c[0]


def _regions(seed):
    regs = []
    for k, name in enumerate(["stream16_r11", "stream16_r04", "stream16_r12"]):
        w = inputs.workload(name)
        regs.append(dict(observed=w["observed"], N_pop=w["P"], eps=w["eps"] * 4.0, pool=1 << 16))
    info, res = abc.abc_smc_run_regions(regs, rounds=4, shrink_rounds=2, sims_per_round=1 << 18, eps_factor=0.7,
                                        flow_blocks=3, flow_hidden=128, train_steps=150, train_steps_warm=60,
                                        train_batch=2048, train_lr=2e-3, seed=seed, mode="fast")
    return _no_times(info), [tuple(t.cpu().numpy() if hasattr(t, "cpu") else t for t in r) for r in res]


def test_per_region_sequential_abc_is_the_same_for_one_seed():
    a, b = _regions(21), _regions(21)
    assert a[0] == b[0]
    assert any(x["proposal"] for x in a[0][-1])
    for ra, rb in zip(a[1], b[1]):
        assert ra[3] == rb[3] and ra[3] > 0
        for x, y in zip(ra[:3], rb[:3]):
            assert np.array_equal(x, y)


def test_population_monte_carlo_is_the_same_for_one_seed():
    """Two population Monte Carlo runs with one seed (region_1e6_T49, four
    rounds of at least 1000 particles): the same rounds, particles, weights and
    distances bit for bit, although the accept slots of each round come from
    atomics in whatever order the batches' warps finish; another seed gives
    another population."""
    w = inputs.workload("region_1e6_T49")
    obs, P = w["observed"], w["P"]
    eps0 = abc.abc_kth_smallest(abc.abc_distances(obs, P, 1 << 18, 99, mode="fast"), 1 << 11)

    def run(seed):
        info, th, wt, dist = abc.abc_pmc_run(obs, P, eps0, rounds=4, n_particles=1000, batch=1 << 16,
                                             max_batches=64, eps_factor=0.7, seed=seed, capacity=1 << 17,
                                             mode="fast")
        return ([(r["n_sims"], r["n_accepted"], r["ess_fraction"]) for r in info], th.cpu().numpy(),
                wt.cpu().numpy(), dist.cpu().numpy())

    a, b, c = run(8), run(8), run(9)
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    assert a[0] != c[0] or not np.array_equal(a[1], c[1])
