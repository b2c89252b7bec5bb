"""abc_sample_async: chunks enqueued back to back on one stream, with the
observed series uploaded once and the counters left on the device, give
exactly the accept sets, counts and simulated days of synchronous abc_sample
calls on the same index ranges (both modes), also when the chunks run as a
captured CUDA graph."""
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


def _sorted(theta, dist, idx):
    o = torch.argsort(idx)
    return theta[o].cpu().numpy(), dist[o].cpu().numpy(), idx[o].cpu().numpy()


def _bufs(k, cap):
    return [(torch.empty((cap, 8), dtype=torch.float32, device=DEV), torch.empty((cap,), dtype=torch.float64, device=DEV),
             torch.empty((cap,), dtype=torch.int64, device=DEV)) for _ in range(k)]


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_async_chunks_equal_sync_calls(mode):
    w = inputs.workload("region_1e7_T60")
    obs = abc.Observed(w["observed"], w["P"])
    d = abc.abc_distances(w["observed"], w["P"], 1 << 16, 77, mode=mode)
    eps = abc.abc_kth_smallest(d, 200)
    k, n, cap = 4, 50000, 4096
    outs = _bufs(k, cap)
    counters = torch.zeros((k, 4), dtype=torch.int64, device=DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for c in range(k):
            abc.abc_sample_async(obs, eps, n, 77, outs[c], counters[c], mode=mode, first_index=c * n + 11,
                                 cuda_stream=s)
    s.synchronize()
    cnt = counters.cpu().numpy()
    for c in range(k):
        ref = abc.abc_sample(w["observed"], w["P"], eps, n, 77, mode=mode, first_index=c * n + 11, capacity=cap)
        days = abc.abc_last_simulated_days()
        assert cnt[c, 0] == ref[3] and cnt[c, 1] >= n and cnt[c, 2] == days
        m = int(cnt[c, 0])
        got = _sorted(outs[c][0][:m], outs[c][1][:m], outs[c][2][:m])
        for a, b in zip(got, _sorted(*ref[:3])):
            assert np.array_equal(a, b)
    obs.close()


def test_async_exact_matches_oracle_and_graph_replay():
    w = inputs.workload("region_1e6_T49")
    obs = abc.Observed(w["observed"], w["P"])
    n = 3000
    ref = oracle.abc(w["observed"], w["P"], 0.0, n, 5, first_index=9, want_all=True, capacity=1)
    eps = float(np.sort(ref["dist_all"])[60])
    want = oracle.abc(w["observed"], w["P"], eps, n, 5, first_index=9, capacity=n)
    out = _bufs(1, 512)[0]
    counters = torch.zeros(3, dtype=torch.int64, device=DEV)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        abc.abc_sample_async(obs, eps, n, 5, out, counters, mode="exact", first_index=9,
                             cuda_stream=torch.cuda.current_stream())
    for _ in range(2):                      # each replay zeroes the counters again
        g.replay()
        torch.cuda.synchronize()
        m = int(counters[0])
        assert m == want["n_accepted"]
        th, di, ix = _sorted(out[0][:m], out[1][:m], out[2][:m])
        assert np.array_equal(ix.astype(np.uint64), want["idx"]) and np.array_equal(th, want["theta"])
        assert np.array_equal(di, want["dist"])
    obs.close()


def test_async_argument_errors():
    w = inputs.workload("region_1e6_T49")
    obs = abc.Observed(w["observed"], w["P"])
    out = _bufs(1, 16)[0]
    with pytest.raises(ValueError):
        abc.abc_sample_async(obs, 1.0, 10, 1, out, torch.zeros(2, dtype=torch.int64, device=DEV))
    with pytest.raises(abc.AbcError):
        abc.abc_sample_async(obs, float("nan"), 10, 1, out, torch.zeros(3, dtype=torch.int64, device=DEV))
    obs.close()
    with pytest.raises(ValueError):
        obs.handle
