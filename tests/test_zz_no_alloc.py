"""The entry point that allocates nothing (abc_sample_noalloc), for callers
that must not allocate device memory while sampling. Through the C ABI, two
calls in a row must return what abc_sample returns for the same inputs: the
same accept count and, sorted by index, bit-identical theta, distances and
indices (the tolerance the exact-mode parity tests use). This file is
collected last so that a run stopping at the first failure has already run
every other test."""
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


def _sorted(theta, dist, idx):
    o = torch.argsort(idx)
    return theta[o].cpu().numpy(), dist[o].cpu().numpy(), idx[o].cpu().numpy()


@pytest.mark.parametrize("name,mode,n", [("region_1e6_T49", "exact", 65536), ("region_6e7_T100", "fast", 1 << 20)])
def test_noalloc_matches_abc_sample_on_two_calls(name, mode, n):
    w = inputs.workload(name)
    obs, P, seed = w["observed"], w["P"], w["seed"]
    eps = w["eps"] if mode == "exact" else w["eps"] * 2.0
    cap = 8192
    th_r, di_r, ix_r, n_r = abc.abc_sample(obs, P, eps, n, seed, mode=mode, capacity=cap)
    ref = _sorted(th_r, di_r, ix_r)
    assert n_r > 0
    out = (torch.empty((cap, 8), dtype=torch.float32, device=DEV), torch.empty((cap,), dtype=torch.float64, device=DEV),
           torch.empty((cap,), dtype=torch.int64, device=DEV))
    for call in range(2):
        th, di, ix, n_acc = abc.abc_sample_noalloc(obs, P, eps, n, seed, out, mode=mode)
        assert n_acc == n_r, call
        got = _sorted(th, di, ix)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), call


def test_noalloc_rejects_horizon_beyond_its_scratch():
    T = abc.binding.ABC_NOALLOC_T_MAX + 1
    obs = np.zeros((3, T + 1), dtype=np.int32)
    obs[0, 0] = 10
    out = (torch.empty((4, 8), dtype=torch.float32, device=DEV), torch.empty((4,), dtype=torch.float64, device=DEV),
           torch.empty((4,), dtype=torch.int64, device=DEV))
    with pytest.raises(abc.AbcError) as e:
        abc.abc_sample_noalloc(obs, 1000, 1.0, 10, 1, out)
    assert e.value.status == abc.binding.ABC_ERR_INVALID_ARG
    assert "no-alloc scratch limit" in e.value.message


def test_noalloc_allocates_nothing(monkeypatch):
    """The property the entry point exists for. With the library's allocation
    paths made to fail (ABC_GB300_INJECT_FAULT=alloc makes every scratch
    allocation return ABC_ERR_NOMEM), abc_sample fails while
    abc_sample_noalloc still succeeds with the same results; and after a
    warm-up call (which loads the kernel's module), two more calls leave the
    device's free memory unchanged to the byte."""
    w = inputs.workload("region_1e6_T49")
    obs, P, seed, eps = w["observed"], w["P"], w["seed"], w["eps"]
    n, cap = 65536, 4096
    out = (torch.empty((cap, 8), dtype=torch.float32, device=DEV), torch.empty((cap,), dtype=torch.float64, device=DEV),
           torch.empty((cap,), dtype=torch.int64, device=DEV))
    ref = _sorted(*abc.abc_sample_noalloc(obs, P, eps, n, seed, out, mode="exact")[:3])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        th, di, ix, _ = abc.abc_sample_noalloc(obs, P, eps, n, seed, out, mode="exact")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    monkeypatch.setenv("ABC_GB300_INJECT_FAULT", "alloc")
    with pytest.raises(abc.AbcError) as e:
        abc.abc_sample(obs, P, eps, n, seed, mode="exact", capacity=cap)
    assert e.value.status == abc.binding.ABC_ERR_NOMEM
    th, di, ix, n_acc = abc.abc_sample_noalloc(obs, P, eps, n, seed, out, mode="exact")
    monkeypatch.delenv("ABC_GB300_INJECT_FAULT")
    for a, b in zip(_sorted(th, di, ix), ref):
        assert np.array_equal(a, b)
