"""Write ``workloads.json``: the synthetic observed series and tolerances of
the benchmark and parity workloads. Calls only the CPU oracle.

The paper fits 49 days of country data that start on the first day with 100
detected cases (Sec. 5); that data is not available here, so each series is
one run of the paper's own stochastic model (Sec. 2.1) at a seeded true theta
from the prior box (Eq. 2), started from (A0, R0, D0) = (100, 0, 0):

  * seed_obs = 20201228 + the workload's position in the table below;
  * theta_true = the first prior draw (seed_obs, stream 2, index j = 0, 1, ...)
    whose trajectory is epidemic-shaped: final A+R+D in [10 A0, P/2], S > 0;
  * observed = that trajectory's (A, R, D) rows, from (seed_obs, stream 1,
    index 0), exact-mode arithmetic;
  * eps = a distance quantile of a pilot batch of prior samples (seed_pilot,
    stream 0), rounded to 3 significant figures (workloads with a fixed eps),
    or the exact quantile of the workload's own batch (the 0.1 % workload).

Run:  python tests/golden/make_workloads.py   (takes about a minute)
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

SEED_OBS = 20201228
SEED_ABC = 1234
SEED_PILOT = 4321
A0 = 100

WORKLOADS = {
    # one region, P = 1e6, T = 49, 65,536 prior samples, eps = 0.1 % quantile, exact mode
    "region_1e6_T49": dict(P=10**6, T=49, n_samples=65536, quantile=0.001, mode="exact"),
    # one region, P = 6e7, T = 100, 2^24 prior samples per launch, eps at ~1e-4 acceptance, fast mode
    "region_6e7_T100": dict(P=6 * 10**7, T=100, n_samples=1 << 24, quantile=1e-4, pilot=1 << 20,
                            mode="fast"),
    # three regions batched, 2^22 samples each, eps at ~1e-4 acceptance each
    "region_1e7_T60": dict(P=10**7, T=60, n_samples=1 << 22, quantile=1e-4, pilot=1 << 20, mode="fast"),
    "region_6e7_T90": dict(P=6 * 10**7, T=90, n_samples=1 << 22, quantile=1e-4, pilot=1 << 20, mode="fast"),
    "region_3p3e8_T120": dict(P=330_000_000, T=120, n_samples=1 << 22, quantile=1e-4, pilot=1 << 20,
                              mode="fast"),
}


# sixteen regions for the streamed batch: populations log-uniform in 1e6 .. 3e8,
# horizons uniform in 30 .. 180 days (seeded), 2^24 / 16 = 2^20 samples each per chunk
def stream_regions():
    g = np.random.default_rng(20210101)
    out = {}
    for r in range(16):
        P = int(round(10 ** g.uniform(6, np.log10(3e8))))
        T = int(g.integers(30, 181))
        out["stream16_r%02d" % r] = dict(P=P, T=T, n_samples=1 << 20, quantile=1e-4, pilot=1 << 18, mode="fast")
    return out


WORKLOADS.update(stream_regions())


def round_sig(x, sig=3):
    if x == 0:
        return 0.0
    return float(round(x, sig - 1 - int(math.floor(math.log10(abs(x))))))


def make(name, spec, seed_obs):
    P, T = spec["P"], spec["T"]
    for j in range(10000):
        th = oracle.prior_draw(seed_obs, 2, j)
        traj = oracle.simulate(th, [A0, 0, 0], T, P, seed_obs, 1, 0)
        final = int(traj[-1, 2:5].sum())
        if 10 * A0 <= final <= P // 2 and traj[-1, 0] > 0:
            break
    else:
        raise RuntimeError("no epidemic-shaped theta found")
    observed = np.ascontiguousarray(traj[:, 2:5].T)
    out = dict(P=P, T=T, n_samples=spec["n_samples"], mode=spec["mode"], seed_obs=seed_obs,
               theta_true_index=j, theta_true=[float(v) for v in th], A0=A0,
               seed=SEED_ABC, stream=0, quantile=spec["quantile"],
               observed=observed.tolist())
    if "pilot" in spec:
        n = spec["pilot"]
        r = oracle.abc(observed, P, 0.0, n, SEED_PILOT, want_all=True, capacity=1)
        k = int(math.ceil(spec["quantile"] * n))
        d = np.sort(r["dist_all"])[k - 1]
        out.update(eps=round_sig(float(d)), pilot=n, seed_pilot=SEED_PILOT, pilot_k=k)
    else:
        n = spec["n_samples"]
        r = oracle.abc(observed, P, 0.0, n, SEED_ABC, want_all=True, capacity=1)
        k = int(math.ceil(spec["quantile"] * n))
        out.update(eps=float(np.sort(r["dist_all"])[k - 1]), quantile_k=k)
    return out


def main():
    res = {}
    for w, (name, spec) in enumerate(WORKLOADS.items()):
        res[name] = make(name, spec, SEED_OBS + w)
        print(name, "theta_true index", res[name]["theta_true_index"], "eps", res[name]["eps"],
              "final ARD", [row[-1] for row in res[name]["observed"]])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
