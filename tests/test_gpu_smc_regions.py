"""Sequential ABC with one learned proposal per region, several regions in one
batched launch per round (abc_smc_run_regions): each region's pooled,
importance-weighted samples at its final tolerance estimate the same ABC
posterior (Eq. 7) as plain rejection from the prior at that tolerance (every
coordinate's mean within 0.05 posterior sd and CDF at five quantiles within
0.02, beyond Monte-Carlo error), and the learned proposals give far more
effective samples per simulation than the prior. Both fallback rules: by ESS
fraction below 10 % (the 16-region stream's stated rule) and by efficiency
against the prior."""
import numpy as np
import pytest

from tests import inputs
from tests.smc_rules import flow_is_kept
from tests.stats_helpers import assert_posterior_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_14332_gb300 as abc  # noqa: E402
from paper_2012_14332_gb300 import build as _build  # noqa: E402

_build.build()
NAMES = ["stream16_r11", "stream16_r15", "stream16_r04", "stream16_r12"]


@pytest.mark.parametrize("rule", ["ess", "efficiency"])
def test_per_region_flows_keep_each_posterior(rule):
    regs = []
    for k, name in enumerate(NAMES):
        w = inputs.workload(name)
        pilot = abc.abc_distances(w["observed"], w["P"], 1 << 20, 300 + k, mode="fast")
        eps = abc.abc_kth_smallest(pilot, 1 << 10)            # ~1e-3 prior acceptance
        regs.append(dict(observed=w["observed"], N_pop=w["P"], eps=eps, pool=1 << 18))
    rounds, shrink, n = 6, 3, 1 << 18
    info, res = abc.abc_smc_run_regions(regs, rounds=rounds, shrink_rounds=shrink, sims_per_round=n, eps_factor=0.7,
                                        flow_blocks=3, flow_hidden=128, train_steps=400, train_steps_warm=150,
                                        train_batch=4096, train_lr=2e-3, seed=21, mode="fast", fallback=rule)
    for r in range(rounds):
        print("round %d: %s" % (r, "  ".join("%d/%d ess %.2f" % (x["proposal"], x["n_accepted"], x["ess_fraction"])
                                             for x in info[r])))
    for g, reg in enumerate(regs):
        th, wt, di, n_pooled = res[g]
        assert n_pooled == sum(info[r][g]["n_accepted"] for r in range(shrink - 1, rounds))
        assert 0 < th.shape[0] <= min(n_pooled, 1 << 18)
        assert np.all(di.cpu().numpy() <= reg["eps"])
        assert info[shrink - 1][g]["eps"] == reg["eps"] and info[0][g]["eps"] > reg["eps"]
        for r in range(rounds - 1):
            # a region may also stay on the prior for want of training points
            assert info[r + 1][g]["proposal"] <= flow_is_kept(info[r][g], 0.1, rule), (g, r)
        used_flow = [info[r][g]["proposal"] for r in range(1, rounds)]
        assert 2 * sum(used_flow) >= len(used_flow), (g, used_flow)
        # plain prior ABC at the same final tolerance
        n_plain = 1 << 25
        th_p, _, _, n_acc_p = abc.abc_sample(reg["observed"], reg["N_pop"], reg["eps"], n_plain, 777 + g, mode="fast",
                                             capacity=1 << 17)
        assert n_acc_p > 2000
        p_prior = n_acc_p / n_plain
        a = th.cpu().numpy().astype(np.float64)
        wa = wt.cpu().numpy()
        wa = wa / wa.sum()
        # what the learned proposals gain: effective pooled samples per
        # simulation at the final eps against the prior's acceptance there
        eff = 1.0 / (wa ** 2).sum()
        per_sim = eff / (n * (rounds - shrink + 1))
        print("region %d: prior acceptance %.3e, pooled effective samples per simulation %.3e, pooled %d" % (
            g, p_prior, per_sim, n_pooled))
        assert per_sim > 3 * p_prior
        b = th_p.cpu().numpy().astype(np.float64)
        assert_posterior_close(a, wa, b, tag="region %d" % g)
