"""Posterior-predictive projections (Sec. 5: accepted samples simulated 120
days forward, 5th to 95th percentile bands): exact-mode bands equal the order
statistics of the oracle's trajectories bit for bit."""
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
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("B", [1, 100, 257, 1000])
def test_bands_equal_oracle_order_statistics(B):
    w = inputs.workload("region_1e6_T49")
    th, _, idx, n = abc.abc_sample(w["observed"], w["P"], 2 * w["eps"], 1 << 18, w["seed"], mode="exact",
                                   capacity=4096)
    assert n >= B
    th, idx = th[:B], idx[:B]
    T = 120
    q = np.array([0.05, 0.25, 0.5, 0.75, 0.95, 0.0, 1.0])
    bands = abc.abc_project(th, idx, w["observed"][:, 0], T, w["P"], w["seed"], quantiles=q,
                            mode="exact").cpu().numpy()
    thn, idn = th.cpu().numpy(), idx.cpu().numpy()
    traj = np.stack([oracle.simulate(thn[b], w["observed"][:, 0], T, w["P"], w["seed"], 0, int(idn[b]))
                     for b in range(B)])
    ard = np.sort(traj[:, :, 2:5], axis=0)
    for k, qq in enumerate(q):
        want = ard[int(np.floor(qq * (B - 1)))].astype(np.float32)
        assert np.array_equal(bands[k], want), (k, qq)
    # the first 49 days of the projection are the accepted trajectories' own days
    assert np.all(bands[0] <= bands[2]) and np.all(bands[2] <= bands[4])
