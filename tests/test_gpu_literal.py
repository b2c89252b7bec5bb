"""The literal-variance model variant (transition standard deviation h^(1/4),
the second reading of Sec. 2.1's "variance sqrt(h)"; ABC_VARIANCE_LITERAL):
exact mode against the oracle's variance_literal path bit for bit (single
steps, trajectories, distances and the accept set); fast mode against exact
mode in distribution; the batched and sequential calls refuse it."""
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


def test_literal_steps_and_trajectories_bit_exact():
    B, P = 6000, 6 * 10**7
    X = inputs.random_states(21, B, P)
    th = inputs.random_thetas(22, B)
    g = inputs.rng(23)
    idx = g.integers(0, 2**33, size=B).astype(np.int64)
    day = g.integers(1, 200, size=B).astype(np.int32)
    Y, n = abc.abc_step(torch.from_numpy(th).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(idx).to(DEV),
                        torch.from_numpy(day).to(DEV), P, 31, stream=4, mode="exact_literal")
    Y, n = Y.cpu().numpy(), n.cpu().numpy()
    Y_std, _ = abc.abc_step(torch.from_numpy(th).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(idx).to(DEV),
                            torch.from_numpy(day).to(DEV), P, 31, stream=4, mode="exact")
    assert not np.array_equal(Y, Y_std.cpu().numpy())      # the variant changes the draws
    for b in range(0, B, 5):
        k = (int(day[b]) + 1) // 2
        z = oracle.day_pair_normals(31, 4, int(idx[b]), k)
        zd = z[:5] if day[b] % 2 == 1 else z[5:]
        n_ref, Y_ref = oracle.step(X[b], th[b], P, zd, variance_literal=True)
        assert np.array_equal(Y[b], Y_ref) and np.array_equal(n[b], n_ref), b
    T = 60
    th2 = oracle.prior_batch(78, 1, 0, 200)
    idx2 = inputs.rng(24).integers(0, 2**40, size=200).astype(np.int64)
    traj = abc.abc_simulate(torch.from_numpy(th2).to(DEV), torch.from_numpy(idx2).to(DEV), [100, 0, 0], T, 10**6, 55,
                            stream=2, mode="exact_literal").cpu().numpy()
    for b in range(200):
        ref = oracle.simulate(th2[b], [100, 0, 0], T, 10**6, 55, 2, int(idx2[b]), variance_literal=True)
        assert np.array_equal(traj[b], ref), b


def test_literal_accept_set_bit_exact():
    w = inputs.workload("region_1e6_T49")
    n = 20000
    ref = oracle.abc(w["observed"], w["P"], 0.0, n, 9, first_index=3, want_all=True, capacity=1,
                     variance_literal=True)
    d = abc.abc_distances(w["observed"], w["P"], n, 9, mode="exact_literal", first_index=3).cpu().numpy()
    assert np.array_equal(d, ref["dist_all"])
    eps = float(np.sort(ref["dist_all"])[200])
    want = oracle.abc(w["observed"], w["P"], eps, n, 9, first_index=3, capacity=n, variance_literal=True)
    th, di, ix, m = abc.abc_sample(w["observed"], w["P"], eps, n, 9, mode="exact_literal", first_index=3,
                                   capacity=4096)
    o = torch.argsort(ix)
    assert m == want["n_accepted"]
    assert np.array_equal(ix[o].cpu().numpy().astype(np.uint64), want["idx"])
    assert np.array_equal(th[o].cpu().numpy(), want["theta"]) and np.array_equal(di[o].cpu().numpy(), want["dist"])


def test_literal_fast_mode_matches_exact_in_distribution():
    """Fast and exact literal samplers draw the same words: their acceptance
    rates at a common eps agree within Monte-Carlo error."""
    w = inputs.workload("region_1e7_T60")
    n = 1 << 22
    d = abc.abc_distances(w["observed"], w["P"], 1 << 18, 5, mode="exact_literal")
    eps = abc.abc_kth_smallest(d, 1 << 8)
    _, _, _, a_fast = abc.abc_sample(w["observed"], w["P"], eps, n, 6, mode="fast_literal", capacity=1 << 16)
    _, _, _, a_exact = abc.abc_sample(w["observed"], w["P"], eps, n, 6, mode="exact_literal", capacity=1 << 16)
    se = np.sqrt(a_exact * 2.0)
    assert abs(a_fast - a_exact) < 5 * se + 5, (a_fast, a_exact)


def test_batched_and_sequential_calls_refuse_the_variant():
    w = inputs.workload("region_1e6_T49")
    with pytest.raises(abc.AbcError):
        abc.Plan([dict(observed=w["observed"], N_pop=w["P"], eps=1e6, n_samples=64)], 1, mode="fast_literal")
    with pytest.raises(abc.AbcError):
        abc.abc_smc_run(w["observed"], w["P"], 1e6, rounds=1, sims_per_round=1024, mode="fast_literal")
