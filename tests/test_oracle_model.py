"""Pins of the oracle's model and ABC loop against what the paper and the
mathematics fix: conservation, non-negativity, the zero-infection fixed point,
special values of Eq. 4, closed-form moments of the floored Gaussian
transitions (Sec. 2.1 third step), the large-population limit (mean
recursion), brute-force acceptance probabilities on tiny populations, the
exact distance (Sec. 2.2) and the batched accept set (Sec. 3.1)."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from tests import inputs

SEED, STREAM = 777, 0


# --------------------------------------------------------------------------
# transition count: floor, clamp
# --------------------------------------------------------------------------
def test_clamp_count_cases():
    cc = oracle.clamp_count
    assert cc(float("nan"), 10) == 0
    assert cc(-5.0, 10) == 0
    assert cc(-0.5, 10) == 0
    assert cc(0.0, 10) == 0
    assert cc(0.999, 10) == 0
    assert cc(3.7, 10) == 3
    assert cc(10.0, 10) == 10
    assert cc(12.0, 10) == 10
    assert cc(float("inf"), 10) == 10
    assert cc(3e9, 2**31 - 1) == 2**31 - 1
    assert cc(5.0, 0) == 0
    # above 2^24 the float already is an integer: n = min(x, c)
    assert cc(float(np.float32(2**24 + 2)), 2**24 + 1) == 2**24 + 1
    assert cc(float(np.float32(2**24 + 2)), 2**30) == 2**24 + 2


# --------------------------------------------------------------------------
# Eq. 4 special values, Eq. 5 structure
# --------------------------------------------------------------------------
def test_infection_rate_special_values():
    th = np.array([0.25, 40.0, 1.3, 0.1, 0.2, 0.05, 0.5, 1.0], dtype=np.float32)
    # U = 0: (A+R+D)^n = 0, so g = alpha0 + alpha
    assert oracle.infection_rate(th, 0) == np.float32(th[0] + th[1])
    # U = 1: 1^n = 1, so g = alpha0 + alpha / 2
    assert oracle.infection_rate(th, 1) == np.float32(th[0] + th[1] / np.float32(2))
    # n = 0: U^0 = 1 for every U >= 1
    th0 = th.copy()
    th0[2] = 0
    for U in (1, 7, 1000, 10**8):
        assert oracle.infection_rate(th0, U) == np.float32(th[0] + th[1] / np.float32(2))
    # non-increasing in U for n > 0, tends to alpha0
    Us = np.unique(np.geomspace(1, 2**31 - 1, 400).astype(np.int64))
    g = np.array([oracle.infection_rate(th, int(U)) for U in Us])
    assert np.all(np.diff(g) <= 0)
    assert abs(g[-1] - th[0]) < 1e-10 * th[1] + 1e-7
    # against the float64 formula: relative error of a float32 pow via exp2(n log2 U)
    for U in Us[::20]:
        ref = th[0] + th[1] / (1 + float(U) ** float(th[2]))
        got = float(oracle.infection_rate(th, int(U)))
        assert abs(got - ref) <= 1e-6 * (abs(ref) + th[1] * 1e-2)


def test_hazard_structure():
    th = np.array([0.25, 40.0, 1.3, 0.1, 0.2, 0.05, 0.5, 1.0], dtype=np.float32)
    P = 10**6
    # no infected: S->I, I->A, I->Ru vanish
    h = oracle.hazard([P - 300, 0, 100, 100, 100, 0], th, P)
    assert h[0] == 0 and h[1] == 0 and h[4] == 0 and h[2] > 0 and h[3] > 0
    # no active cases: A->R, A->D vanish
    h = oracle.hazard([P - 100, 100, 0, 0, 0, 0], th, P)
    assert h[2] == 0 and h[3] == 0 and h[0] > 0
    # ratios fixed by Eq. 5: h5 / h2 = beta eta / gamma, h3 / h4 = beta / delta
    h = oracle.hazard([P - 5000, 2000, 1000, 1000, 500, 500], th, P)
    assert h[4] / h[1] == pytest.approx(th[3] * th[6] / th[4], rel=1e-6)
    assert h[2] / h[3] == pytest.approx(th[3] / th[5], rel=1e-6)
    # S -> I is bilinear in S and I: g S I / P
    g = oracle.infection_rate(th, 2500)
    assert h[0] == pytest.approx(float(g) * (P - 5000) * 2000 / P, rel=1e-6)
    assert h[1] == pytest.approx(th[4] * 2000, rel=1e-7)


# --------------------------------------------------------------------------
# closed-form moments of one transition
# --------------------------------------------------------------------------
def _count_pmf(h, c):
    """P(n = j), j = 0..c, for n = min(max(floor(h + sqrt(h) Z), 0), c)."""
    if c == 0 or h <= 0:
        p = np.zeros(c + 1)
        p[0] = 1.0
        return p
    s = math.sqrt(h)
    j = np.arange(c + 1, dtype=np.float64)
    upper = stats.norm.cdf((j + 1 - h) / s)
    lower = stats.norm.cdf((j - h) / s)
    p = upper - lower
    p[0] = upper[0]
    p[c] = 1.0 - lower[c]
    return p


def _expected_counts(h, X):
    S, I, A = int(X[0]), int(X[1]), int(X[2])
    out = np.zeros((5, 2))
    for k, c in ((0, S), (1, I), (2, A)):
        p = _count_pmf(float(h[k]), c)
        j = np.arange(c + 1)
        out[k] = (p @ j, p @ j**2)
    # chained caps: I -> Ru limited by I - n(I->A), A -> D by A - n(A->R)
    for k, first, src in ((4, 1, I), (3, 2, A)):
        p_first = _count_pmf(float(h[first]), src)
        m1 = m2 = 0.0
        for j1, pj in enumerate(p_first):
            if pj < 1e-18:
                continue
            c = src - j1
            p = _count_pmf(float(h[k]), c)
            j = np.arange(c + 1)
            m1 += pj * (p @ j)
            m2 += pj * (p @ j**2)
        out[k] = (m1, m2)
    return out


@pytest.mark.parametrize("case", range(4))
def test_transition_moments_match_closed_form(case):
    """Mean and variance of each of the five counts, drawn with independent
    N(0,1) normals, against the exact floored/clamped Gaussian sums."""
    states = [
        ([900, 60, 30, 5, 3, 2], 1000),
        ([5_000_000, 40_000, 9_000, 700, 100, 200], 5_050_000),
        ([12, 3, 2, 0, 0, 1], 18),
        ([400, 7, 50, 10, 2, 1], 470),
    ]
    thetas = [
        [0.3, 5.0, 0.5, 0.2, 0.3, 0.05, 0.6, 1.0],
        [0.5, 20.0, 1.2, 0.05, 0.15, 0.01, 0.9, 1.0],
        [0.9, 1.0, 1.0, 0.5, 0.6, 0.3, 0.9, 1.0],
        [0.2, 80.0, 0.3, 0.9, 0.95, 0.8, 0.99, 1.0],
    ]
    X = np.array(states[case][0], dtype=np.int32)
    P = states[case][1]
    th = np.array(thetas[case], dtype=np.float32)
    m = 200_000
    z = inputs.rng(100 + case).standard_normal((m, 5)).astype(np.float32)
    n, Y = oracle.step_batch(np.tile(X, (m, 1)), np.tile(th, (m, 1)), P, z)
    h = oracle.hazard(X, th, P)
    ex = _expected_counts(h, X)
    for k in range(5):
        mean, m2 = ex[k]
        var = max(m2 - mean**2, 1e-12)
        assert abs(n[:, k].mean() - mean) < 5 * math.sqrt(var / m) + 1e-9, (k, n[:, k].mean(), mean)
        if var > 1e-6:
            assert abs(n[:, k].var() / var - 1) < 5 * math.sqrt(2 / m) * 3, (k, n[:, k].var(), var)


def test_variance_literal_reading():
    """x = h + h^(1/4) z under the literal reading of 'variance sqrt(h)'."""
    X = np.array([10**7 - 11000, 10000, 1000, 0, 0, 0], dtype=np.int32)
    th = np.array([0.3, 0.0, 1.0, 0.1, 0.4, 0.05, 0.5, 1.0], dtype=np.float32)
    P = 10**7
    m = 100_000
    z = inputs.rng(4).standard_normal((m, 5)).astype(np.float32)
    Xs, ths = np.tile(X, (m, 1)), np.tile(th, (m, 1))
    n_std, _ = oracle.step_batch(Xs, ths, P, z, variance_literal=False)
    n_lit, _ = oracle.step_batch(Xs, ths, P, z, variance_literal=True)
    h = oracle.hazard(X, th, P).astype(np.float64)
    assert n_std[:, 1].var() == pytest.approx(h[1] + 1 / 12, rel=0.03)
    assert n_lit[:, 1].var() == pytest.approx(math.sqrt(h[1]) + 1 / 12, rel=0.03)


# --------------------------------------------------------------------------
# trajectories: invariants and fixed points
# --------------------------------------------------------------------------
def test_conservation_and_nonnegativity():
    g = inputs.rng(21)
    thetas = oracle.prior_batch(SEED, 5, 0, 60)
    for j, th in enumerate(thetas):
        P = int(g.choice([1000, 10**6, 6 * 10**7, 330_000_000]))
        A0 = int(g.integers(0, min(P // 3, 10**5) + 1))
        ard0 = [A0, int(g.integers(0, A0 + 1)), int(g.integers(0, A0 // 10 + 1))]
        traj = oracle.simulate(th, ard0, 120, P, SEED, STREAM, j).astype(np.int64)
        assert np.all(traj >= 0)
        assert np.all(traj.sum(axis=1) == P)
        assert np.all(np.diff(traj[:, 0]) <= 0)                  # S only drains
        assert np.all(np.diff(traj[:, 3:6], axis=0) >= 0)        # R, D, Ru only fill
        assert traj[0, 5] == 0 and list(traj[0, 2:5]) == ard0     # initial condition


def test_zero_infection_fixed_point():
    th = np.array([0.9, 50.0, 1.0, 0.3, 0.5, 0.1, 0.7, 0.0], dtype=np.float32)   # kappa = 0
    traj = oracle.simulate(th, [0, 0, 0], 60, 10**6, SEED, STREAM, 3)
    assert np.all(traj == np.array([10**6, 0, 0, 0, 0, 0]))
    # I = 0 but A > 0: only A drains into R and D
    traj = oracle.simulate(th, [5000, 10, 2], 60, 10**6, SEED, STREAM, 4).astype(np.int64)
    assert np.all(traj[:, 0] == 10**6 - 5012) and np.all(traj[:, 1] == 0) and np.all(traj[:, 5] == 0)
    assert np.all(traj[:, 2:5].sum(axis=1) == 5012)
    assert traj[-1, 2] < 5000


def test_initial_condition_kappa():
    th = oracle.prior_draw(SEED, 0, 0)
    th[7] = 1.5
    X = oracle.init_state(th, [200, 30, 4], 10**5)
    assert list(X) == [10**5 - 234 - 300, 300, 200, 30, 4, 0]
    # I0 limited by the remaining population
    X = oracle.init_state(th, [200, 30, 4], 400)
    assert list(X) == [0, 166, 200, 30, 4, 0]
    with pytest.raises(ValueError):
        oracle.init_state(th, [200, 30, 4], 100)


def _mean_recursion(th, x0, P, T):
    """Deterministic limit: X_{t+1} = X_t + stoichiometry (h(X_t) - 1/2) in
    float64 (E floor(h + sqrt(h) Z) -> h - 1/2 for large h)."""
    a0, a, nexp, b, gam, dl, eta, kap = [float(v) for v in th]
    S, I, A, R, D, Ru = [float(v) for v in x0]
    out = [[S, I, A, R, D, Ru]]
    for _ in range(T):
        U = A + R + D
        g = a0 + a / (1 + U**nexp)
        h = [g * S * I / P - 0.5, gam * I - 0.5, b * A - 0.5, dl * A - 0.5, b * eta * I - 0.5]
        S, I, A, R, D, Ru = (S - h[0], I + h[0] - h[1] - h[4], A + h[1] - h[2] - h[3], R + h[2], D + h[3],
                             Ru + h[4])
        out.append([S, I, A, R, D, Ru])
    return np.array(out)


def test_large_population_limit():
    """Trajectories / P converge to the mean recursion as P grows; the gap
    shrinks about like 1/sqrt(P)."""
    th = np.array([0.35, 0.0, 1.0, 0.08, 0.15, 0.01, 0.5, 2.0], dtype=np.float32)
    T = 40
    errs = {}
    for P in (10**6, 10**8):
        A0 = P // 1000
        ard0 = [A0, A0 // 10, A0 // 100]
        e = []
        for i in range(8):
            traj = oracle.simulate(th, ard0, T, P, SEED, STREAM, i).astype(np.float64)
            ref = _mean_recursion(th, traj[0], P, T)
            e.append(np.max(np.abs(traj - ref)) / P)
        errs[P] = float(np.mean(e))
    # early fluctuations are amplified by the growth phase, so the gap at a
    # given P is ~0.1/sqrt(P) of the population; its ratio is what scales
    assert errs[10**8] < 2e-3
    assert 5.0 < errs[10**6] / errs[10**8] < 20.0, errs


# --------------------------------------------------------------------------
# distance (Sec. 2.2, Eq. 7) and the ABC loop (Sec. 2.2, Sec. 3.1)
# --------------------------------------------------------------------------
def test_sq_distance_exact_and_saturating():
    g = inputs.rng(8)
    T = 37
    traj = g.integers(0, 2**31 - 1, size=(T + 1, 6)).astype(np.int32)
    obs = g.integers(0, 2**31 - 1, size=(3, T + 1)).astype(np.int32)
    exact = sum((int(traj[d, 2 + c]) - int(obs[c, d])) ** 2 for d in range(1, T + 1) for c in range(3))
    assert oracle.sq_distance(traj, obs) == min(exact, 2**63)
    assert exact > 2**63  # this case saturates
    traj = g.integers(0, 10**6, size=(T + 1, 6)).astype(np.int32)
    obs = g.integers(0, 10**6, size=(3, T + 1)).astype(np.int32)
    exact = sum((int(traj[d, 2 + c]) - int(obs[c, d])) ** 2 for d in range(1, T + 1) for c in range(3))
    assert oracle.sq_distance(traj, obs) == exact
    # day 0 never counts
    obs2 = obs.copy()
    obs2[:, 0] += 12345
    assert oracle.sq_distance(traj, obs2) == exact
    for acc in (0, 1, 2, 10**15, 2**53 + 1, 2**63):
        assert oracle.distance_from_sq(acc) == math.sqrt(float(acc))


def _small_observed(P, T, seed):
    th = np.array([0.4, 3.0, 1.0, 0.3, 0.5, 0.1, 0.5, 1.0], dtype=np.float32)
    return np.ascontiguousarray(oracle.simulate(th, [3, 1, 0], T, P, seed, 9, 0)[:, 2:5].T)


@pytest.mark.parametrize("P,eps", [(10, 2.5), (12, 3.2), (8, 1.5)])
def test_acceptance_probability_brute_force(P, eps):
    """P(dist <= eps | theta) by enumerating every transition vector of a
    two-day simulation on a tiny population, against the Monte-Carlo
    acceptance rate of the oracle's ABC loop with a point-mass prior."""
    T = 2
    obs = _small_observed(P, T, 5)
    th = np.array([0.8, 2.0, 0.7, 0.35, 0.6, 0.15, 0.7, 0.9], dtype=np.float32)
    X0 = oracle.init_state(th, obs[:, 0], P)

    def day(X):
        h = oracle.hazard(X, th, P)
        S, I, A = int(X[0]), int(X[1]), int(X[2])
        p1, p2, p3 = _count_pmf(h[0], S), _count_pmf(h[1], I), _count_pmf(h[2], A)
        for n1, n2, n3 in itertools.product(range(S + 1), range(I + 1), range(A + 1)):
            q = p1[n1] * p2[n2] * p3[n3]
            if q < 1e-16:
                continue
            p5 = _count_pmf(h[4], I - n2)
            p4 = _count_pmf(h[3], A - n3)
            for n5, n4 in itertools.product(range(I - n2 + 1), range(A - n3 + 1)):
                qq = q * p5[n5] * p4[n4]
                if qq < 1e-16:
                    continue
                Y = np.array([X[0] - n1, X[1] + n1 - n2 - n5, X[2] + n2 - n3 - n4, X[3] + n3, X[4] + n4,
                              X[5] + n5], dtype=np.int32)
                yield qq, Y

    p_acc = 0.0
    for q1, X1 in day(X0):
        d1 = sum((int(X1[2 + c]) - int(obs[c, 1])) ** 2 for c in range(3))
        for q2, X2 in day(X1):
            d2 = sum((int(X2[2 + c]) - int(obs[c, 2])) ** 2 for c in range(3))
            if math.sqrt(d1 + d2) <= eps:
                p_acc += q1 * q2
    n = 200_000
    r = oracle.abc(obs, P, eps, n, 4242, lo=th, hi=th, capacity=n)
    rate = r["n_accepted"] / n
    sd = math.sqrt(max(p_acc * (1 - p_acc), 1e-9) / n)
    assert 0.01 < p_acc < 0.99
    assert abs(rate - p_acc) < 5 * sd + 2e-4, (rate, p_acc)


def test_abc_accept_set_is_the_filtered_batch():
    """Sec. 3.1: the batched accept set is exactly {i : dist_i <= eps}, with
    theta_i the prior draw of i; independent of threading and of sharding."""
    P, T = 10**6, 30
    obs = np.ascontiguousarray(oracle.simulate(oracle.prior_draw(1, 2, 3), [100, 0, 0], T, P, 1, 1, 0)[:, 2:5].T)
    n = 20_000
    full = oracle.abc(obs, P, 0.0, n, SEED, want_all=True, n_threads=1)
    eps = float(np.sort(full["dist_all"])[40])
    a = oracle.abc(obs, P, eps, n, SEED, want_all=True, n_threads=1)
    b = oracle.abc(obs, P, eps, n, SEED, n_threads=7)
    want = np.nonzero(a["dist_all"] <= eps)[0]
    assert a["n_accepted"] == len(want) >= 41
    assert np.array_equal(a["idx"], want)
    assert np.array_equal(a["dist"], a["dist_all"][want])
    assert np.array_equal(a["theta"], oracle.prior_batch(SEED, 0, 0, n)[want])
    for key in ("idx", "theta", "dist"):
        assert np.array_equal(a[key], b[key])
    lo = oracle.abc(obs, P, eps, n // 2, SEED, first_index=0)
    hi = oracle.abc(obs, P, eps, n - n // 2, SEED, first_index=n // 2)
    assert np.array_equal(np.concatenate([lo["idx"], hi["idx"]]), a["idx"])
    # distances equal the distance of the replayed trajectory
    for i, d in zip(a["idx"][:5], a["dist"][:5]):
        traj = oracle.simulate(oracle.prior_draw(SEED, 0, int(i)), obs[:, 0], T, P, SEED, 0, int(i))
        assert oracle.distance_from_sq(oracle.sq_distance(traj, obs)) == d
    # capacity overflow reports the true count
    c = oracle.abc(obs, P, eps, n, SEED, capacity=5)
    assert c["overflow"] and c["n_accepted"] == a["n_accepted"] and np.array_equal(c["idx"], a["idx"][:5])
