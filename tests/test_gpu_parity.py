"""GPU parity: the CUDA library through its C ABI against the CPU oracle on
the same seeded inputs. Exact mode must agree bit for bit: prior draws, the
Philox words (also against cuRAND), trajectories, single steps, every
distance, the accept set and the eps quantile. All are checked at sizes that
span many blocks with a ragged tail, at every workload shape, and on sampled
outputs at the full 2^24-sample launch the benchmark times."""
import ctypes
import os
import subprocess

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
SHAPES = ["region_1e6_T49", "region_6e7_T100", "region_1e7_T60", "region_6e7_T90", "region_3p3e8_T120"]


def _sorted(theta, dist, idx):
    o = torch.argsort(idx)
    return (theta[o].cpu().numpy(), dist[o].cpu().numpy(), idx[o].cpu().numpy().astype(np.uint64))


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------
_CURAND_SRC = r"""
#include <cstdint>
#include <curand_kernel.h>
__global__ void k(const uint4* c, const uint2* key, uint4* out, int n) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = curand_Philox4x32_10(c[j], key[j]);
}
extern "C" int curand_philox_blocks(const void* c, const void* key, void* out, int n) {
    k<<<(n + 127) / 128, 128>>>((const uint4*)c, (const uint2*)key, (uint4*)out, n);
    return (int)cudaDeviceSynchronize();
}
"""


def test_philox_words_match_curand_and_oracle():
    """The library's Philox (seen through the prior draw: theta_j = lo_j +
    width_j u(w_j) with lo = 0, width = 1 gives u(w_j) itself) against
    cuRAND's Philox4x32-10 block function and the oracle."""
    build_dir = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
    os.makedirs(build_dir, exist_ok=True)
    src = os.path.join(build_dir, "curand_pin.cu")
    so = os.path.join(build_dir, "libcurand_pin.so")
    with open(src, "w") as f:
        f.write(_CURAND_SRC)
    subprocess.check_call([_build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, src])
    lib = ctypes.CDLL(so)
    seed, stream, n = 0x0123456789ABCDEF, 5, 3000
    first = (1 << 32) - 1000
    c = np.zeros((2 * n, 4), dtype=np.uint32)
    i = np.arange(first, first + n, dtype=np.uint64)
    for g in range(2):
        c[g::2, 0] = (i & 0xFFFFFFFF).astype(np.uint32)
        c[g::2, 1] = (i >> 32).astype(np.uint32)
        c[g::2, 2] = 0
        c[g::2, 3] = (stream << 2) | g
    key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (2 * n, 1))
    cd, kd = torch.from_numpy(c.view(np.int32)).to(DEV), torch.from_numpy(key.view(np.int32)).to(DEV)
    out = torch.zeros((2 * n, 4), dtype=torch.int32, device=DEV)
    assert lib.curand_philox_blocks(ctypes.c_void_p(cd.data_ptr()), ctypes.c_void_p(kd.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), 2 * n) == 0
    words = out.cpu().numpy().view(np.uint32).reshape(n, 8)
    # oracle words
    for j in (0, 1, 999, 1000, n - 1):
        ow = np.concatenate([oracle.philox4x32_10(c[2 * j + g], key[0]) for g in range(2)])
        assert np.array_equal(ow, words[j])
    # library words through the unit box
    obs = np.zeros((3, 3), dtype=np.int32)
    obs[0, 0] = 10
    _, th = abc.abc_distances(obs, 1000, n, seed, stream=stream, mode="exact", first_index=first,
                              lo=np.zeros(8), hi=np.ones(8), want_theta=True)
    u_ref = oracle.uniform_batch(words.ravel()).reshape(n, 8)
    assert np.array_equal(th.cpu().numpy(), u_ref)


@pytest.mark.parametrize("first", [0, 12345, (1 << 32) - 777, (1 << 40) + 3])
def test_prior_draws_bit_exact(first):
    n = 5000
    obs = inputs.workload("region_1e6_T49")["observed"]
    _, th = abc.abc_distances(obs, 10**6, n, 1234, stream=3, mode="fast", first_index=first, want_theta=True)
    assert np.array_equal(th.cpu().numpy(), oracle.prior_batch(1234, 3, first, n))


# --------------------------------------------------------------------------
# trajectories and single steps
# --------------------------------------------------------------------------
@pytest.mark.parametrize("P,T", [(10**6, 49), (6 * 10**7, 100), (330_000_000, 120), (1000, 31), (1, 5),
                                 (10**5, 1)])
def test_trajectories_bit_exact(P, T):
    B = 300
    g = inputs.rng(P % 1000 + T)
    th = oracle.prior_batch(77, 1, 0, B)
    th[:10, 7] = 0.0                        # no initial infected
    th[10:20, 2] = 0.0                      # n = 0
    idx = g.integers(0, 2**40, size=B).astype(np.int64)
    A0 = min(100, P)
    init = [A0, 0, 0]
    traj = abc.abc_simulate(torch.from_numpy(th).to(DEV), torch.from_numpy(idx).to(DEV), init, T, P, 55,
                            stream=2, mode="exact").cpu().numpy()
    for b in range(B):
        ref = oracle.simulate(th[b], init, T, P, 55, 2, int(idx[b]))
        assert np.array_equal(traj[b], ref), b


def test_steps_bit_exact_on_random_states():
    """abc_step against oracle.step with the oracle's own normals of the same
    (sample, day): the whole day (Eq. 4, Eq. 5, floored counts, clamps)."""
    B = 20000
    P = 6 * 10**7
    X = inputs.random_states(8, B, P)
    X[:2000, 1] = 0                                     # zero-infection rows ...
    X[:2000, 0] = P - X[:2000, 2:].sum(axis=1)          # ... still summing to P
    th = inputs.random_thetas(9, B)
    g = inputs.rng(10)
    idx = g.integers(0, 2**33, size=B).astype(np.int64)
    day = g.integers(1, 200, size=B).astype(np.int32)
    Y, n = abc.abc_step(torch.from_numpy(th).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(idx).to(DEV),
                        torch.from_numpy(day).to(DEV), P, 31, stream=4, mode="exact")
    Y, n = Y.cpu().numpy(), n.cpu().numpy()
    for b in range(0, B, 7):
        k = (int(day[b]) + 1) // 2
        z = oracle.day_pair_normals(31, 4, int(idx[b]), k)
        zd = z[:5] if day[b] % 2 == 1 else z[5:]
        n_ref, Y_ref = oracle.step(X[b], th[b], P, zd)
        assert np.array_equal(Y[b], Y_ref) and np.array_equal(n[b], n_ref), b
    assert np.all(Y.astype(np.int64).sum(axis=1) == P) and np.all(Y >= 0)


# --------------------------------------------------------------------------
# distances, accept sets, quantile
# --------------------------------------------------------------------------
def test_region_1e6_T49_full_exact():
    """The 0.1 %-quantile workload in full (65,536 samples): every distance,
    the eps quantile and the accept set bit-equal to the oracle."""
    w = inputs.workload("region_1e6_T49")
    obs, P, n, seed = w["observed"], w["P"], w["n_samples"], w["seed"]
    ref = oracle.abc(obs, P, 0.0, n, seed, want_all=True, capacity=1)
    d = abc.abc_distances(obs, P, n, seed, mode="exact")
    assert np.array_equal(d.cpu().numpy(), ref["dist_all"])
    k = w["quantile_k"]
    eps = abc.abc_kth_smallest(d, k)
    assert eps == np.sort(ref["dist_all"])[k - 1] == w["eps"]
    want = oracle.abc(obs, P, eps, n, seed, capacity=n)
    theta, dist, idx, n_acc = abc.abc_sample(obs, P, eps, n, seed, mode="exact", capacity=4096)
    assert n_acc == want["n_accepted"] >= k
    th, di, ix = _sorted(theta, dist, idx)
    assert np.array_equal(ix, want["idx"]) and np.array_equal(th, want["theta"]) and np.array_equal(di, want["dist"])
    # replaying an accepted (theta, idx) reproduces its distance
    traj = abc.abc_simulate(torch.from_numpy(th).to(DEV), torch.from_numpy(ix.astype(np.int64)).to(DEV),
                            obs[:, 0], w["T"], P, seed, mode="exact").cpu().numpy()
    for b in range(len(ix)):
        assert oracle.distance_from_sq(oracle.sq_distance(traj[b], obs)) == di[b]


@pytest.mark.parametrize("name", SHAPES)
def test_every_shape_exact_distances_and_accepts(name):
    """Each workload's shape (P, T, observed series) at 12,345 samples (many
    blocks, ragged tail), exact mode: distances and accept set bit-equal."""
    w = inputs.workload(name)
    obs, P = w["observed"], w["P"]
    n, seed, first = 12345, 2024, 7 * 10**9
    ref = oracle.abc(obs, P, 0.0, n, seed, first_index=first, want_all=True, capacity=1)
    d = abc.abc_distances(obs, P, n, seed, mode="exact", first_index=first)
    assert np.array_equal(d.cpu().numpy(), ref["dist_all"])
    eps = float(np.sort(ref["dist_all"])[60])
    want = oracle.abc(obs, P, eps, n, seed, first_index=first, capacity=n)
    theta, dist, idx, n_acc = abc.abc_sample(obs, P, eps, n, seed, mode="exact", first_index=first, capacity=1024)
    th, di, ix = _sorted(theta, dist, idx)
    assert n_acc == want["n_accepted"]
    assert np.array_equal(ix, want["idx"]) and np.array_equal(th, want["theta"]) and np.array_equal(di, want["dist"])


def test_edge_cases():
    w = inputs.workload("region_1e6_T49")
    obs, P = w["observed"], w["P"]
    # single sample, samples < one warp, exactly one block, one past a block
    for n in (1, 17, 256, 257):
        ref = oracle.abc(obs, P, 0.0, n, 9, first_index=(1 << 32) - 3, want_all=True, capacity=1)
        d = abc.abc_distances(obs, P, n, 9, mode="exact", first_index=(1 << 32) - 3)
        assert np.array_equal(d.cpu().numpy(), ref["dist_all"]), n
    # zero samples
    theta, dist, idx, n_acc = abc.abc_sample(obs, P, 1e9, 0, 9, mode="exact")
    assert n_acc == 0 and theta.shape[0] == 0
    # eps = 0 accepts only exact matches: none here
    _, _, _, n_acc = abc.abc_sample(obs, P, 0.0, 4096, 9, mode="exact")
    assert n_acc == 0
    # eps large: everything accepted; capacity overflow reports the true count
    with pytest.raises(abc.AbcError) as e:
        abc.abc_sample(obs, P, 1e30, 3000, 9, mode="exact", capacity=100)
    assert e.value.status == abc.binding.ABC_ERR_CAPACITY
    theta, dist, idx, n_acc = abc.abc_sample(obs, P, 1e30, 3000, 9, mode="exact", capacity=100, allow_overflow=True)
    assert n_acc == 3000 and theta.shape[0] == 100
    assert len(set(idx.cpu().numpy().tolist())) == 100
    # nothing is rejected early when everything is accepted
    assert abc.abc_last_simulated_days() == 3000 * w["T"]
    # early rejection simulates fewer days, never more
    abc.abc_sample(obs, P, w["eps"], 3000, 9, mode="exact")
    assert 0 < abc.abc_last_simulated_days() < 3000 * w["T"]
    # capacity zero with accepts
    _, _, _, n_acc = abc.abc_sample(obs, P, 1e30, 50, 9, mode="exact", capacity=0, allow_overflow=True)
    assert n_acc == 50
    # degenerate box: every theta equal to lo
    lo = np.array([0.3, 20, 1.0, 0.2, 0.3, 0.05, 0.5, 1.0], dtype=np.float32)
    _, th = abc.abc_distances(obs, P, 600, 9, mode="exact", lo=lo, hi=lo, want_theta=True)
    assert np.all(th.cpu().numpy() == lo)


# P = 2^31 - 1 with 10^9 initially active: the daily differences reach 2^31,
# so sums of squares cross 2^62 and 2^63. Series "mixed" puts about half the
# samples between 2^62 and 2^63 and some past 2^63; in "day_past_2_63" the
# three squares of day 1 alone exceed 2^63 (they still fit in 64 bits).
P_TOP = 2**31 - 1


def _top_range_observed(kind):
    obs = np.zeros((3, 3), dtype=np.int32)
    obs[:, 0] = [10**9, 0, 0]
    if kind == "mixed":
        obs[:, 1] = obs[:, 2] = [0, 2 * 10**9, 10**9]
    else:
        obs[:, 1] = [0, P_TOP, P_TOP]
        obs[:, 2] = [0, 0, 0]
    return obs


@pytest.mark.parametrize("kind", ["mixed", "day_past_2_63"])
def test_distance_at_the_top_of_its_range(kind):
    """Eq. 7 with the exact uint64 sum saturating at 2^63: every distance
    (abc_distances) equals the oracle's, including sqrt(2^63) for saturated
    sums; the accept sets of abc_reject_kernel (abc_sample) and of
    abc_batch_kernel (a one-region plan) equal the oracle's at an eps just
    below 2^31 (threshold below 2^62: the kernels' clamped accumulation), at
    an eps whose threshold lies between 2^62 and 2^63 (accepted sums in that
    range) and at eps = sqrt(2^63) (saturated sums accepted too)."""
    obs = _top_range_observed(kind)
    n, seed = 20000, 77
    ref = oracle.abc(obs, P_TOP, 0.0, n, seed, want_all=True, capacity=1)
    d_all = ref["dist_all"]
    top = float(np.sqrt(np.float64(2.0**63)))
    d = abc.abc_distances(obs, P_TOP, n, seed, mode="exact").cpu().numpy()
    assert np.array_equal(d, d_all)
    n_sat, n_mid = int(np.sum(d_all == top)), int(np.sum((d_all >= 2.0**31) & (d_all < top)))
    print("%s: %d saturated, %d between 2^62 and 2^63, %d below" % (kind, n_sat, n_mid, n - n_sat - n_mid))
    assert n_sat > 0
    if kind == "mixed":
        assert n_mid > 0.2 * n and n - n_sat - n_mid > 0.2 * n
    else:
        # day 1's three squares alone pass 2^63 for some saturated samples (oracle trajectories, exact integers)
        past = 0
        for i in np.flatnonzero(d_all == top)[:100]:
            traj = oracle.simulate(oracle.prior_draw(seed, 0, int(i)), obs[:, 0], 2, P_TOP, seed, 0, int(i))
            past += sum((int(traj[1, 2 + c]) - int(obs[c, 1])) ** 2 for c in range(3)) >= 2**63
        assert past > 0
    for eps in (2.0**31 - 0.5, float(np.sort(d_all)[int(0.75 * n)]), top):
        want = oracle.abc(obs, P_TOP, eps, n, seed, capacity=n)
        if eps > 2.0**31 and eps < top:
            assert np.sum(want["dist"] >= 2.0**31) > 1000
        theta, dist, idx, n_acc = abc.abc_sample(obs, P_TOP, eps, n, seed, mode="exact", capacity=n)
        th, di, ix = _sorted(theta, dist, idx)
        assert n_acc == want["n_accepted"], eps
        assert np.array_equal(ix, want["idx"]) and np.array_equal(th, want["theta"]) and np.array_equal(di, want["dist"])
        plan = abc.Plan([dict(observed=obs, N_pop=P_TOP, eps=eps, n_samples=n, first_index=0, stream=0, capacity=n)],
                        seed, mode="exact")
        plan.run()
        th, di, ix, n_acc, _ = plan.results(0)
        th, di, ix = _sorted(th, di, ix)
        plan.close()
        assert n_acc == want["n_accepted"], eps
        assert np.array_equal(ix, want["idx"]) and np.array_equal(th, want["theta"]) and np.array_equal(di, want["dist"])


def test_long_horizons_in_turn():
    """Kernels whose shared memory passes 48 KB at long horizons (the
    rejection kernel from T = 1792, the distance kernel from T = 3072) run at
    T = 4000, then 2000 or 3100, then 4000 again: a shorter horizon must not
    lower the kernel's shared-memory limit under a longer one launched before."""
    g = inputs.rng(5)
    for T_mid in (2000, 3100):
        for T in (4000, T_mid, 4000):
            obs = np.zeros((3, T + 1), dtype=np.int32)
            obs[:, 1:] = g.integers(0, 300, size=(3, T))
            obs[:, 0] = [50, 5, 1]
            n = 96
            ref = oracle.abc(obs, 10**4, 0.0, n, 3, want_all=True, capacity=1)
            d = abc.abc_distances(obs, 10**4, n, 3, mode="exact")
            assert np.array_equal(d.cpu().numpy(), ref["dist_all"]), T
            eps = float(np.sort(ref["dist_all"])[n // 4])
            want = oracle.abc(obs, 10**4, eps, n, 3, capacity=n)
            theta, dist, idx, n_acc = abc.abc_sample(obs, 10**4, eps, n, 3, mode="exact", capacity=n)
            th, di, ix = _sorted(theta, dist, idx)
            assert n_acc == want["n_accepted"], T
            assert np.array_equal(ix, want["idx"]) and np.array_equal(di, want["dist"]), T


def test_longest_horizon_and_tiny_population():
    """T = ABC_T_MAX (64 KiB of shared memory per block) and P = 1."""
    T = abc.ABC_T_MAX
    g = inputs.rng(1)
    obs = np.zeros((3, T + 1), dtype=np.int32)
    obs[:, 1:] = g.integers(0, 500, size=(3, T))
    obs[:, 0] = [50, 5, 1]
    n = 700
    ref = oracle.abc(obs, 10**4, 0.0, n, 3, want_all=True, capacity=1)
    d = abc.abc_distances(obs, 10**4, n, 3, mode="exact")
    assert np.array_equal(d.cpu().numpy(), ref["dist_all"])
    obs1 = np.zeros((3, 8), dtype=np.int32)
    obs1[0, 0] = 1
    ref = oracle.abc(obs1, 1, 0.0, 300, 3, want_all=True, capacity=1)
    d = abc.abc_distances(obs1, 1, 300, 3, mode="exact")
    assert np.array_equal(d.cpu().numpy(), ref["dist_all"])


def test_kth_smallest_matches_sort():
    """The radix select against a sort (ties, zeros, 1e300 and +inf
    included), from a pass of one block with a ragged tail to passes of many
    blocks, where the last block to finish each pass picks its digit."""
    g = inputs.rng(2)
    x = np.concatenate([g.random(100_003) * 1e6, [0.0, 0.0, 5.0, 5.0, 1e300, np.inf]])
    big = np.concatenate([x, g.random(200_000) * 1e3, x[:5000]])
    for n in (7, 200, len(x), 1 << 17, (1 << 17) + 1, len(big)):
        v = big[:n]
        t = torch.from_numpy(v).to(DEV)
        vs = np.sort(v)
        for k in sorted({1, 2, 3, 50, n // 2, n - 1, n} & set(range(1, n + 1))):
            assert abc.abc_kth_smallest(t, k) == vs[k - 1]


@pytest.mark.parametrize("bad", [np.nan, -1.0, -0.0, -np.inf])
def test_kth_smallest_rejects_values_that_do_not_order(bad):
    """A NaN, a negative value or -0 would sort by its bit pattern above
    every distance: the call refuses the input instead of returning a wrong
    quantile."""
    for n in (5000, 200_000):   # the one-block and the many-block form
        x = inputs.rng(6).random(n) * 100.0
        x[1234] = bad
        with pytest.raises(abc.AbcError) as e:
            abc.abc_kth_smallest(torch.from_numpy(x).to(DEV), 10)
        assert e.value.status == abc.binding.ABC_ERR_INVALID_ARG
        x[1234] = 0.0
        assert abc.abc_kth_smallest(torch.from_numpy(x).to(DEV), 1) == 0.0


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_select_below_equals_rejection_at_eps(mode):
    """The quantile pipeline of the small workload (P = 1e6, T = 49, 65,536
    prior samples): every distance with theta, eps as the 66-th smallest
    distance (0.1 %), then the samples at or below eps selected from those
    distances. The selected (index, theta, distance) set equals the rejection
    launch's at that eps bit for bit, in both modes (a mode's distances are the
    same in both calls); in exact mode it is also the oracle's accept set."""
    w = inputs.workload("region_1e6_T49")
    obs, P, n, seed = w["observed"], w["P"], w["n_samples"], w["seed"]
    d, th_all = abc.abc_distances(obs, P, n, seed, mode=mode, first_index=7, want_theta=True)
    eps = abc.abc_kth_smallest(d, 66)
    th, di, ix, m = abc.abc_select_below(d, eps, first_index=7, theta=th_all, capacity=1024)
    assert m >= 66
    ref = abc.abc_sample(obs, P, eps, n, seed, mode=mode, first_index=7, capacity=1024)
    assert ref[3] == m
    a, b = _sorted(th, di, ix), _sorted(*ref[:3])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    if mode == "exact":
        res = oracle.abc(obs, P, eps, n, seed, first_index=7)
        assert np.array_equal(a[2], np.asarray(res["idx"], dtype=np.uint64))
        assert np.array_equal(a[1], np.asarray(res["dist"], dtype=np.float64))
    # capacity below the count: the true count, and the call reports it
    with pytest.raises(abc.AbcError) as e:
        abc.abc_select_below(d, eps, first_index=7, theta=th_all, capacity=m - 1)
    assert e.value.status == abc.binding.ABC_ERR_CAPACITY
    # without theta: indices and distances only
    none, di2, ix2, m2 = abc.abc_select_below(d, eps, first_index=7, capacity=1024)
    assert none is None and m2 == m
    o = np.argsort(ix2.cpu().numpy())
    assert np.array_equal(ix2.cpu().numpy()[o], a[2]) and np.array_equal(di2.cpu().numpy()[o], a[1])


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_sample_quantile_equals_the_three_calls(mode):
    """abc_sample_quantile, the one-call form of the quantile pipeline, on the
    small workload (P = 1e6, T = 49, 65,536 samples, k = 66): the same eps and
    the same accepted (index, theta, distance) set as abc_distances,
    abc_kth_smallest and abc_select_below in turn; in exact mode eps is the
    oracle-written workload's and the set is the oracle's. Then the edges:
    k = 1 (the minimum), k = n (every sample, eps the largest distance), a
    ragged n with an offset first index, and a capacity below the count."""
    w = inputs.workload("region_1e6_T49")
    obs, P, n, seed = w["observed"], w["P"], w["n_samples"], w["seed"]
    th, di, ix, m, eps = abc.abc_sample_quantile(obs, P, n, 66, seed, mode=mode, capacity=1024)
    d, th_all = abc.abc_distances(obs, P, n, seed, mode=mode, want_theta=True)
    assert eps == abc.abc_kth_smallest(d, 66)
    ref = abc.abc_select_below(d, eps, theta=th_all, capacity=1024)
    assert m == ref[3] >= 66
    a, b = _sorted(th, di, ix), _sorted(*ref[:3])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    if mode == "exact":
        assert eps == w["eps"]
        want = oracle.abc(obs, P, eps, n, seed, capacity=n)
        assert m == want["n_accepted"]
        assert np.array_equal(a[2], np.asarray(want["idx"], dtype=np.uint64))
        assert np.array_equal(a[0], want["theta"]) and np.array_equal(a[1], want["dist"])
    dn = np.sort(d.cpu().numpy())
    _, di1, _, m1, e1 = abc.abc_sample_quantile(obs, P, n, 1, seed, mode=mode, capacity=16)
    assert e1 == dn[0] and m1 == int(np.count_nonzero(dn == dn[0])) and di1.cpu().numpy()[0] == dn[0]
    n2, first = 3001, 10**10 + 5
    _, _, ix2, m2, e2 = abc.abc_sample_quantile(obs, P, n2, n2, seed, mode=mode, first_index=first, capacity=n2)
    d2 = abc.abc_distances(obs, P, n2, seed, mode=mode, first_index=first).cpu().numpy()
    assert e2 == d2.max() and m2 == n2
    assert np.array_equal(np.sort(ix2.cpu().numpy().astype(np.uint64)), first + np.arange(n2, dtype=np.uint64))
    with pytest.raises(abc.AbcError) as e:
        abc.abc_sample_quantile(obs, P, n, 66, seed, mode=mode, capacity=m - 1)
    assert e.value.status == abc.binding.ABC_ERR_CAPACITY


def test_scratch_pool_reuses_its_memory():
    """Calls that take stream-ordered scratch reuse the pool's memory: ten
    one-call quantile runs over 2^20 samples (40 MB of scratch each) leave the
    device's free memory within 256 MB of where it was after the first, and
    give the same result every time."""
    w = inputs.workload("region_6e7_T100")
    obs, P, seed = w["observed"], w["P"], w["seed"]
    n, k = 1 << 20, 100
    out = (torch.empty((4096, 8), dtype=torch.float32, device=DEV), torch.empty((4096,), dtype=torch.float64, device=DEV),
           torch.empty((4096,), dtype=torch.int64, device=DEV))
    first = abc.abc_sample_quantile(obs, P, n, k, seed, mode="fast", out=out)
    ref = (first[3], first[4], np.sort(first[2].cpu().numpy()))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(10):
        r = abc.abc_sample_quantile(obs, P, n, k, seed, mode="fast", out=out)
        assert (r[3], r[4]) == ref[:2] and np.array_equal(np.sort(r[2].cpu().numpy()), ref[2])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 256 << 20


def test_local_k_smallest_for_the_distributed_quantile():
    """A rank's part of the distributed quantile (sharding.local_k_smallest):
    its k smallest distances, found on the device by the radix select and the
    accept step, equal the first k of a sort; ties at the k-th value (more
    of them than k) and k above n are handled."""
    from paper_2012_14332_gb300.sharding import local_k_smallest
    w = inputs.workload("region_1e6_T49")
    d = abc.abc_distances(w["observed"], w["P"], 20000, w["seed"], mode="exact", first_index=3)
    ref = np.sort(d.cpu().numpy())
    for k in (1, 66, 1000):
        assert np.array_equal(local_k_smallest(d, k), ref[:k])
    x = np.concatenate([np.full(300, 2.5), inputs.rng(9).random(5000) * 10 + 3.0, [0.5, 1.0]])
    t = torch.from_numpy(x).to(DEV)
    assert np.array_equal(local_k_smallest(t, 10), np.sort(x)[:10])
    assert np.array_equal(local_k_smallest(t[:50], 80), np.full(50, 2.5))


def test_full_size_launch_sampled_against_oracle():
    """The benchmark's launch: 2^24 samples of the P = 6e7, T = 100 workload.
    Exact mode: every accepted sample is re-derived by the oracle (theta bits,
    distance bits), and a random subset of indices is classified by the oracle
    and must be accepted exactly when the oracle accepts it. Fast mode: the
    accepted theta are the oracle's prior draws of their indices."""
    w = inputs.workload("region_6e7_T100")
    obs, P, T, n, seed, eps = w["observed"], w["P"], w["T"], w["n_samples"], w["seed"], w["eps"]
    cap = 1 << 16
    theta, dist, idx, n_acc = abc.abc_sample(obs, P, eps, n, seed, mode="exact", capacity=cap)
    th, di, ix = _sorted(theta, dist, idx)
    assert 0.2e-4 * n < n_acc < 5e-4 * n
    acc_set = set(ix.tolist())
    pick = inputs.rng(3).choice(len(ix), size=min(64, len(ix)), replace=False)
    for b in pick:
        i = int(ix[b])
        t_ref = oracle.prior_draw(seed, 0, i)
        assert np.array_equal(th[b], t_ref)
        traj = oracle.simulate(t_ref, obs[:, 0], T, P, seed, 0, i)
        assert oracle.distance_from_sq(oracle.sq_distance(traj, obs)) == di[b] <= eps
    probe = inputs.rng(4).integers(0, n, size=3000)
    for i in probe:
        traj = oracle.simulate(oracle.prior_draw(seed, 0, int(i)), obs[:, 0], T, P, seed, 0, int(i))
        d = oracle.distance_from_sq(oracle.sq_distance(traj, obs))
        assert (d <= eps) == (int(i) in acc_set), i
    theta, dist, idx, n_fast = abc.abc_sample(obs, P, eps, n, seed, mode="fast", capacity=cap)
    th, di, ix = _sorted(theta, dist, idx)
    assert abs(n_fast - n_acc) < 6 * np.sqrt(n_acc) + 10
    for b in range(0, len(ix), max(1, len(ix) // 64)):
        assert np.array_equal(th[b], oracle.prior_draw(seed, 0, int(ix[b])))
        assert di[b] <= eps
