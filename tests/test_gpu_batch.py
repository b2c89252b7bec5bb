"""Batched regions (abc_plan_*): one persistent launch over a table of regions
with their own population, horizon, eps, observed series, random stream and
sample range must give, region by region, exactly the accept sets of the
oracle (exact mode) and of abc_sample (both modes); runs advance the sample
ranges, CUDA-graph replays equal plain runs, proposal buffers replace the
prior draw, and the autotuner leaves the plan's state unchanged."""
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
NAMES = ["region_1e7_T60", "region_6e7_T90", "region_3p3e8_T120", "region_1e6_T49"]
SEED = 4711


def _sorted(theta, dist, idx):
    o = torch.argsort(idx)
    return theta[o].cpu().numpy(), dist[o].cpu().numpy(), idx[o].cpu().numpy().astype(np.uint64)


def _regions(n_list, first_list, quantile=0.01):
    regs = []
    for r, (name, n, first) in enumerate(zip(NAMES, n_list, first_list)):
        w = inputs.workload(name)
        ref = oracle.abc(w["observed"], w["P"], 0.0, max(n, 1), SEED, stream=10 + r, first_index=first,
                         want_all=True, capacity=1)
        eps = float(np.sort(ref["dist_all"])[int(quantile * max(n, 1))]) if n else 1e6
        regs.append(dict(observed=w["observed"], N_pop=w["P"], eps=eps, n_samples=n, first_index=first,
                         stream=10 + r, capacity=4096))
    return regs


def test_plan_exact_matches_oracle_per_region():
    regs = _regions([6000, 7001, 5003, 0], [0, 10**9, (1 << 32) - 100, 5])
    plan = abc.Plan(regs, SEED, mode="exact")
    plan.run()
    for r, g in enumerate(regs):
        want = oracle.abc(g["observed"], g["N_pop"], g["eps"], g["n_samples"], SEED, stream=g["stream"],
                          first_index=g["first_index"], capacity=max(g["n_samples"], 1))
        th, di, ix, n_acc, days = plan.results(r)
        th, di, ix = _sorted(th, di, ix)
        assert n_acc == want["n_accepted"], r
        assert np.array_equal(ix, want["idx"]) and np.array_equal(th, want["theta"]) and np.array_equal(di, want["dist"])
        if g["n_samples"]:
            assert 0 < days <= g["n_samples"] * (g["observed"].shape[1] - 1)
    plan.close()


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_plan_equals_abc_sample_and_runs_advance(mode):
    n = 40000
    regs = _regions([n, n, n], [0, 777, 123456])
    plan = abc.Plan(regs, SEED, mode=mode)
    plan.run()
    plan.run()
    for r, g in enumerate(regs):
        ref = abc.abc_sample(g["observed"], g["N_pop"], g["eps"], 2 * n, SEED, stream=g["stream"], mode=mode,
                             first_index=g["first_index"], capacity=4096)
        days_ref = abc.abc_last_simulated_days()
        th, di, ix, n_acc, days = plan.results(r)
        assert n_acc == ref[3]
        assert days == days_ref
        for a, b in zip(_sorted(th, di, ix), _sorted(*ref[:3])):
            assert np.array_equal(a, b)
    plan.close()


def test_graph_replay_equals_runs():
    n = 30000
    regs = _regions([n, n // 3, n], [0, 50, 99])
    a = abc.Plan(regs, SEED, mode="fast")
    for _ in range(3):
        a.run()
    b = abc.Plan(regs, SEED, mode="fast")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run_graph(3, cuda_stream=s)
    s.synchronize()
    for r in range(len(regs)):
        ra, rb = a.results(r), b.results(r)
        assert ra[3] == rb[3] and ra[4] == rb[4]
        for x, y in zip(_sorted(*ra[:3]), _sorted(*rb[:3])):
            assert np.array_equal(x, y)
    a.close()
    b.close()


def test_plan_with_proposal_buffer():
    """theta_in replaces the prior draw: sample j of the run gets theta_in[j]
    and the random numbers of index first_index + j."""
    w = inputs.workload("region_1e6_T49")
    n, first, stream = 3000, 222, 7
    th = inputs.random_thetas(12, n)
    th[:, 1] *= 0.1                                 # a narrower proposal than the prior
    th_d = torch.from_numpy(th).to(DEV)
    d = np.array([oracle.distance_from_sq(oracle.sq_distance(
        oracle.simulate(th[j], w["observed"][:, 0], w["T"], w["P"], SEED, stream, first + j), w["observed"]))
        for j in range(n)])
    eps = float(np.sort(d)[150])
    plan = abc.Plan([dict(observed=w["observed"], N_pop=w["P"], eps=eps, n_samples=n, first_index=first,
                          stream=stream, capacity=n, theta_in=th_d)], SEED, mode="exact")
    plan.run()
    tt, di, ix, n_acc, _ = plan.results(0)
    tt, di, ix = _sorted(tt, di, ix)
    want = np.nonzero(d <= eps)[0]
    assert n_acc == len(want)
    assert np.array_equal(ix, want + first) and np.array_equal(di, d[want]) and np.array_equal(tt, th[want])
    plan.close()


def test_several_regions_with_proposal_buffers_match_oracle():
    """Three regions, each with its own proposal buffer, in one plan (their
    series staged in shared memory): each region's accept set equals the
    oracle's over its proposals, bit for bit in exact mode."""
    names = ["region_1e6_T49", "region_1e7_T60", "region_6e7_T90"]
    regs, want = [], []
    for r, name in enumerate(names):
        w = inputs.workload(name)
        n, first, stream = 1500 + 37 * r, 1000 * r + 5, 30 + r
        th = inputs.random_thetas(40 + r, n)
        th[:, 2] *= 0.5                                 # proposals away from the prior
        d = np.array([oracle.distance_from_sq(oracle.sq_distance(
            oracle.simulate(th[j], w["observed"][:, 0], w["T"], w["P"], SEED, stream, first + j), w["observed"]))
            for j in range(n)])
        eps = float(np.sort(d)[40 + 10 * r])
        regs.append(dict(observed=w["observed"], N_pop=w["P"], eps=eps, n_samples=n, first_index=first,
                         stream=stream, capacity=n, theta_in=torch.from_numpy(th).to(DEV)))
        want.append((th, d, eps, first))
    plan = abc.Plan(regs, SEED, mode="exact")
    plan.run()
    for r, (th, d, eps, first) in enumerate(want):
        tt, di, ix, n_acc, _ = plan.results(r)
        tt, di, ix = _sorted(tt, di, ix)
        keep = np.nonzero(d <= eps)[0]
        assert n_acc == len(keep), r
        assert np.array_equal(ix, keep.astype(np.uint64) + first) and np.array_equal(di, d[keep])
        assert np.array_equal(tt, th[keep])
    plan.close()


def test_tune_keeps_state_and_picks_a_shape():
    n = 1 << 18
    regs = _regions([n, n, n], [0, 0, 0])
    plan = abc.Plan(regs, SEED, mode="fast")
    plan.run()
    before = [plan.counts(r) for r in range(3)]
    best, shapes = plan.tune()
    assert len(shapes) >= 6 and best["ms"] == min(s["ms"] for s in shapes)
    assert [plan.counts(r) for r in range(3)] == before
    plan.run()
    for r, g in enumerate(regs):
        ref = abc.abc_sample(g["observed"], g["N_pop"], g["eps"], 2 * n, SEED, stream=g["stream"], mode="fast",
                             first_index=g["first_index"], capacity=8192)
        assert plan.counts(r)[0] == ref[3]
    plan.close()


def test_nan_proposals_are_skipped():
    w = inputs.workload("region_1e6_T49")
    n, first, stream = 2000, 10, 3
    th = inputs.random_thetas(13, n)
    skip = np.zeros(n, dtype=bool)
    skip[::3] = True
    skip[1500:1540] = True
    th_nan = th.copy()
    th_nan[skip, 0] = np.nan
    eps = 1e12   # accept every simulated sample
    plan = abc.Plan([dict(observed=w["observed"], N_pop=w["P"], eps=eps, n_samples=n, first_index=first,
                          stream=stream, capacity=n, theta_in=torch.from_numpy(th_nan).to(DEV))], SEED, mode="exact")
    plan.run()
    tt, di, ix, n_acc, days = plan.results(0)
    tt, di, ix = _sorted(tt, di, ix)
    keep = np.nonzero(~skip)[0]
    assert n_acc == len(keep) and np.array_equal(ix, keep + first) and np.array_equal(tt, th[keep])
    assert days == len(keep) * w["T"]
    plan.close()


def test_chunks_of_skipped_proposals_do_not_end_the_run():
    """A warp that claims a chunk of 32 skipped (NaN) proposals while all its
    lanes are idle must claim again rather than stop: here every chunk but
    the last is skipped, and there are more chunks than resident warps, so
    each warp's first claims find nothing to run."""
    w = inputs.workload("region_1e6_T49")
    n, first, stream = 32 * 60000, 77, 4
    th = inputs.random_thetas(14, n)
    th_nan = th.copy()
    th_nan[:-32, 0] = np.nan
    plan = abc.Plan([dict(observed=w["observed"], N_pop=w["P"], eps=1e12, n_samples=n, first_index=first,
                          stream=stream, capacity=64, theta_in=torch.from_numpy(th_nan).to(DEV))], SEED, mode="fast")
    plan.run()
    tt, di, ix, n_acc, days = plan.results(0)
    tt, di, ix = _sorted(tt, di, ix)
    assert n_acc == 32 and days == 32 * w["T"]
    assert np.array_equal(ix, np.arange(n - 32, n, dtype=np.uint64) + first) and np.array_equal(tt, th[-32:])
    plan.close()


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_long_series_read_through_the_cache_equal_abc_sample(mode):
    """Regions whose observed series together exceed what the kernel stages in
    shared memory (2048 days) are read through the read-only cache; each
    region's accept set still equals abc_sample's. The series are the
    oracle's trajectories of seeded draws over 1100 days."""
    regs = []
    for r, (P, seed) in enumerate([(10 ** 6, 31), (5 * 10 ** 6, 32)]):
        T = 1100
        th = inputs.random_thetas(seed, 1)[0]
        traj = oracle.simulate(th, [100, 0, 0], T, P, seed, 1, 0)
        obs = np.ascontiguousarray(traj[:, 2:5].T).astype(np.int32)
        regs.append(dict(observed=obs, N_pop=P, eps=0.0, n_samples=3000, first_index=17, stream=20 + r,
                         capacity=3000))
    for g in regs:
        d = abc.abc_distances(g["observed"], g["N_pop"], g["n_samples"], SEED, stream=g["stream"], mode=mode,
                              first_index=g["first_index"]).cpu().numpy()
        g["eps"] = float(np.sort(d)[60])
    plan = abc.Plan(regs, SEED, mode=mode)
    plan.run()
    for r, g in enumerate(regs):
        ref = abc.abc_sample(g["observed"], g["N_pop"], g["eps"], g["n_samples"], SEED, stream=g["stream"], mode=mode,
                             first_index=g["first_index"], capacity=3000)
        res = plan.results(r)
        assert res[3] == ref[3] >= 61
        for x, y in zip(_sorted(*res[:3]), _sorted(*ref[:3])):
            assert np.array_equal(x, y)
    plan.close()


def test_graph_follows_an_eps_change_across_2_to_the_62():
    """The batched kernel has a cheaper distance accumulation for thresholds
    below 2^62; a graph captured with it is recaptured when set_eps moves a
    region's threshold past 2^62 (eps >= 2^31), so replays stay exact."""
    w = inputs.workload("region_1e6_T49")
    n = 4096
    reg = dict(observed=w["observed"], N_pop=w["P"], eps=1e4, n_samples=n, first_index=0, stream=2, capacity=n)
    a = abc.Plan([reg], SEED, mode="exact")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a.run_graph(1, cuda_stream=s)
        s.synchronize()
        a.reset(s)
        a.set_region(0, None, 0)
        a.set_eps(0, 2.0 ** 40)
        a.run_graph(1, cuda_stream=s)
        s.synchronize()
    b = abc.Plan([dict(reg, eps=2.0 ** 40)], SEED, mode="exact")
    b.run()
    ra, rb = a.results(0), b.results(0)
    assert ra[3] == rb[3] == n
    for x, y in zip(_sorted(*ra[:3]), _sorted(*rb[:3])):
        assert np.array_equal(x, y)
    a.close()
    b.close()


@pytest.mark.parametrize("mode", ["fast", "exact"])
def test_every_launch_shape_gives_the_same_results(mode):
    """Each compiled launch shape, the register-lean form included (fast mode
    only; refused in exact mode), run on the same sample ranges gives the
    same accepted samples per region and the same simulated-day counts."""
    n = 20000
    regs = _regions([n, n + 7, n - 5], [3, 10**9, (1 << 32) - 100], quantile=0.05)
    plan = abc.Plan(regs, SEED, mode=mode)
    _, shapes = plan.tune()
    assert any(s["lean"] for s in shapes) == (mode == "fast")
    ref = None
    for sh in shapes:
        plan.set_shape(sh)
        plan.reset()
        for r, g in enumerate(regs):
            plan.set_region(r, None, g["first_index"])
        plan.run()
        got = []
        for r in range(len(regs)):
            th, di, ix, n_acc, days = plan.results(r)
            got.append((n_acc, days) + _sorted(th, di, ix))
        if ref is None:
            ref = got
            assert all(g[0] > 0 for g in got)
            continue
        for a, b in zip(got, ref):
            assert a[:2] == b[:2], sh
            for x, y in zip(a[2:], b[2:]):
                assert np.array_equal(x, y), sh
    if mode == "exact":
        with pytest.raises(abc.AbcError):
            plan.set_shape(dict(block_threads=256, pairs_per_iteration=2, blocks_per_sm=0, lean=1))
    with pytest.raises(abc.AbcError):
        plan.set_shape(dict(block_threads=96, pairs_per_iteration=1, blocks_per_sm=0, lean=0))
    plan.close()
