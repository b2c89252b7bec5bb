"""Sequential ABC with the learned flow proposal against plain prior ABC at
the same final tolerance: the learned proposal must accept far more of its
simulations (what the trained network gains), while its importance-weighted
accepted samples estimate the same ABC posterior (Eq. 7) as plain rejection
from the prior: every coordinate's weighted mean within 0.05 posterior sd and
its weighted CDF at five quantiles within 0.02 of plain ABC's, beyond
Monte-Carlo error (sandwich standard errors)."""
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


def test_learned_proposal_gains_and_keeps_the_posterior():
    w = inputs.workload("region_1e6_T49")
    obs, P = w["observed"], w["P"]
    pilot = abc.abc_distances(obs, P, 1 << 20, 99, mode="fast")
    eps0 = abc.abc_kth_smallest(pilot, 1 << 13)          # ~0.8 % prior acceptance in round 0
    rounds, N = 4, 1 << 20
    info, th, wt, dist = abc.abc_smc_run(obs, P, eps0, rounds=rounds, sims_per_round=N, eps_factor=0.7,
                                         flow_blocks=3, flow_hidden=128, train_steps=400, train_batch=1024,
                                         train_lr=2e-3, seed=5, mode="fast")
    for r in info:
        print("round eps %.4g proposal %d accepted %d / %d  ESS %.3f  loss %.3f" % (
            r["eps"], r["proposal"], r["n_accepted"], r["n_sims"], r["ess_fraction"], r["train_loss"]))
    eps_f = info[-1]["eps"]
    assert info[0]["proposal"] == 0 and info[-1]["proposal"] == 1
    for r in range(rounds - 1):
        assert info[r + 1]["proposal"] == flow_is_kept(info[r], 0.1), r
    assert all(r["ess_fraction"] > 0.1 for r in info)
    # plain prior ABC at the final tolerance
    n_plain = 1 << 26
    th_p, _, _, n_acc_p = abc.abc_sample(obs, P, eps_f, n_plain, 12345, mode="fast", capacity=1 << 18)
    p_prior = n_acc_p / n_plain
    p_flow = info[-1]["n_accepted"] / N
    ess = info[-1]["ess_fraction"]
    print("final eps %.4g: prior acceptance %.3e, flow acceptance %.3e (ESS fraction %.3f)" % (eps_f, p_prior, p_flow,
                                                                                                 ess))
    assert n_acc_p > 500
    assert p_flow * ess > 5 * p_prior
    # the weighted flow posterior against plain ABC: every coordinate's mean
    # within 0.05 plain sd and its CDF at five quantiles within 0.02, beyond
    # Monte-Carlo error (four sandwich standard errors)
    a = th.cpu().numpy().astype(np.float64)
    wa = wt.cpu().numpy()
    b = th_p.cpu().numpy().astype(np.float64)
    assert_posterior_close(a, wa, b, tag="learned proposal")
