"""Rejection until a target number of accepts (abc_sample_until): whole
batches of consecutive indices run until the accepted count reaches the
target, and the accepted set is exactly the oracle's over the indices used
(exact mode, bit for bit); max_samples cuts the last batch; an overflow of
the output capacity stops the loop with the true counts."""
import numpy as np
import pytest

import oracle
from tests import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_14332_gb300 as abc  # noqa: E402
from paper_2012_14332_gb300 import build as _build  # noqa: E402

_build.build()
SEED, STREAM, FIRST = 31, 5, (1 << 32) - 5000


def _sorted(theta, dist, idx):
    o = torch.argsort(idx)
    return theta[o].cpu().numpy(), dist[o].cpu().numpy(), idx[o].cpu().numpy().astype(np.uint64)


@pytest.fixture(scope="module")
def setup():
    w = inputs.workload("region_1e6_T49")
    n_all = 16000
    ref = oracle.abc(w["observed"], w["P"], 0.0, n_all, SEED, stream=STREAM, first_index=FIRST, want_all=True,
                     capacity=1)
    eps = float(np.sort(ref["dist_all"])[int(0.004 * n_all)])
    return w, eps, ref["dist_all"]


def test_stops_at_the_first_whole_batch_reaching_the_target(setup):
    w, eps, dist_all = setup
    batch, target = 3000, 30
    cum = np.cumsum(dist_all <= eps)
    k = next(j for j in range(1, len(dist_all) // batch + 1) if cum[j * batch - 1] >= target)
    obs = abc.Observed(w["observed"], w["P"])
    th, di, ix, n_acc, n_used = abc.abc_sample_until(obs, eps, target, SEED, batch=batch, stream=STREAM, mode="exact",
                                                     first_index=FIRST, capacity=1024)
    assert n_used == k * batch and n_acc == cum[n_used - 1] >= target
    want = oracle.abc(w["observed"], w["P"], eps, n_used, SEED, stream=STREAM, first_index=FIRST, capacity=n_used)
    th, di, ix = _sorted(th, di, ix)
    assert np.array_equal(ix, want["idx"]) and np.array_equal(th, want["theta"]) and np.array_equal(di, want["dist"])
    assert 0 < abc.abc_last_simulated_days() <= n_used * w["T"]
    obs.close()


def test_max_samples_cuts_the_last_batch_and_fast_mode_equals_abc_sample(setup):
    w, eps, dist_all = setup
    obs = abc.Observed(w["observed"], w["P"])
    th, di, ix, n_acc, n_used = abc.abc_sample_until(obs, eps, 10 ** 9, SEED, batch=3000, max_samples=7001,
                                                     stream=STREAM, mode="exact", first_index=FIRST, capacity=1024)
    assert n_used == 7001 and n_acc == int(np.sum(dist_all[:7001] <= eps))
    for mode in ("exact", "fast"):
        a = abc.abc_sample_until(obs, eps, 25, SEED, batch=2048, stream=STREAM, mode=mode, first_index=FIRST,
                                 capacity=1024)
        b = abc.abc_sample(w["observed"], w["P"], eps, a[4], SEED, stream=STREAM, mode=mode, first_index=FIRST,
                           capacity=1024)
        assert a[3] == b[3] >= 25 and a[4] % 2048 == 0
        for x, y in zip(_sorted(*a[:3]), _sorted(*b[:3])):
            assert np.array_equal(x, y)
    obs.close()


def test_capacity_overflow_stops_with_true_counts(setup):
    w, eps, dist_all = setup
    obs = abc.Observed(w["observed"], w["P"])
    cum = np.cumsum(dist_all <= eps)
    with pytest.raises(abc.AbcError):
        abc.abc_sample_until(obs, eps, 60, SEED, batch=1000, stream=STREAM, mode="exact", first_index=FIRST,
                             capacity=8)
    _, _, _, n_acc, n_used = abc.abc_sample_until(obs, eps, 60, SEED, batch=1000, stream=STREAM, mode="exact",
                                                  first_index=FIRST, capacity=8, allow_overflow=True)
    k = next(j for j in range(1, 17) if cum[j * 1000 - 1] > 8)
    assert n_used == k * 1000 and n_acc == cum[n_used - 1]
    # nothing to do: no launch, zero counts
    assert abc.abc_sample_until(obs, eps, 0, SEED, mode="exact")[3:] == (0, 0)
    obs.close()
