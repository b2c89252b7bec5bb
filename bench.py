"""Benchmark: ABC rejection sampling on synthetic series shaped like the paper's
country data (Sec. 4, Sec. 5), one JSON line on stdout.

One step = one abc_sample launch over 2^24 prior samples of the P = 6e7,
T = 100 workload at its fixed eps (fast mode), each step on fresh sample
indices. Default: 1 GPU, 10 timed steps after 3 warm-up steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one rank per GPU; ranks take disjoint sample index
ranges (weak scaling, no data-path collective). --impl reference times the CPU
oracle (the plain restatement of the method) on the host cores instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "region_6e7_T100"
METRIC = "accepted ABC samples/s at fixed \u03b5 (learned vs prior proposal); sims\u00b7days/s"
UNIT = "accepted samples/s"

# Algorithmic work of one simulated day (fast mode), in instructions per thread:
# Philox 1.5 blocks x 10 rounds x (2 wide multiplies + 2 three-input xors),
# less the words the three blocks of a day pair share (53); uniforms (7.5);
# 2.5 Box-Muller pairs of 9 (22.5); hazards incl. the pow and four int->float
# (19); five transitions of sqrt, fma, floor, clamp plus two caps (22); state
# update (7); exact distance (11); loop (2). 144 issue slots, 18 of them SFU
# transcendentals. Issue: 4 warp-instructions (128 threads) per clock per SM;
# SFU: 16 per clock per SM.
OPS_PER_SIM_DAY = {"issue": 144.0, "sfu": 18.0}
PIPE_RATE_PER_SM_CLK = {"issue": 128.0, "sfu": 16.0}
# Algorithmic work of one sample besides its days (fast mode): the prior draw,
# two Philox blocks of 10 rounds less the products their shared counter words
# share (73), eight uniforms (16) and the prior's affine map (8); the derived
# rates alpha0/P, alpha/P, beta*eta (3); I0 = floor(kappa A0) clamped and S0 (4).
# 104 issue slots, no SFU transcendental: 104/144 of a simulated day's issue.
OPS_PER_SAMPLE = {"issue": 104.0, "sfu": 0.0}


def load_workload():
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        w = json.load(f)[WORKLOAD]
    w["observed"] = np.array(w["observed"], dtype=np.int32)
    return w


def describe(w):
    return ("%s: one synthetic region, P=%d, T=%d days, %d uniform prior samples per launch, fixed eps=%g "
            "(1e-4 quantile of a %d-sample pilot), %s mode" % (WORKLOAD, w["P"], w["T"], w["n_samples"], w["eps"],
                                                               w["pilot"], w["mode"]))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


# dram__bytes_read.sum + dram__bytes_write.sum per headline launch, taken by
# ncu from a capture of the rejection kernel as it stands; None when the
# kernel has changed since the last capture (the line then reports null).
REJECT_TRAFFIC_BYTES = 153088


def roofline(sim_days_per_launch, launch_ms, sm_count, sm_max_mhz, traffic=None, samples_per_launch=0):
    """ALU roofline: the fastest a launch could run if the tighter of issue
    slots and SFU throughput for the method's instructions were saturated on
    every SM at the maximum SM clock. In simulated days/s: the days the launch
    actually simulated, plus each sample's own work (OPS_PER_SAMPLE) counted
    in days of the bound pipe. days_only_frac leaves the per-sample work out."""
    clk_per_sim_day = max(OPS_PER_SIM_DAY[k] / PIPE_RATE_PER_SM_CLK[k] for k in OPS_PER_SIM_DAY)
    bound_pipe = max(OPS_PER_SIM_DAY, key=lambda k: OPS_PER_SIM_DAY[k] / PIPE_RATE_PER_SM_CLK[k])
    peak = sm_count * sm_max_mhz * 1e6 / clk_per_sim_day
    day_equiv = OPS_PER_SAMPLE[bound_pipe] / OPS_PER_SIM_DAY[bound_pipe]
    days = sim_days_per_launch + day_equiv * samples_per_launch
    achieved = days / (launch_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gsim*days/s",
            "frac": achieved / peak, "traffic": traffic, "pipe": bound_pipe,
            "days_only_frac": sim_days_per_launch / (launch_ms * 1e-3) / peak,
            "peak_basis": "%d SMs x %.0f MHz / %.3f clk per sim-day (%s); a sample's own work = %.3f day" % (
                sm_count, sm_max_mhz, clk_per_sim_day, bound_pipe, day_equiv)}


BATCH_REGIONS = ["region_1e7_T60", "region_6e7_T90", "region_3p3e8_T120"]


def bench_batched(abc, torch, steps, warmup, dev, flush, sm_count, sm_max):
    """Three regions (P = 1e7, 6e7, 3.3e8; T = 60, 90, 120; own eps each; 2^22
    prior samples per region) in one persistent launch per step, replayed from
    a CUDA graph, launch shape from the autotuner."""
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        wl = json.load(f)
    regs = []
    for r, name in enumerate(BATCH_REGIONS):
        w = wl[name]
        regs.append(dict(observed=np.array(w["observed"], dtype=np.int32), N_pop=w["P"], eps=w["eps"],
                         n_samples=w["n_samples"], first_index=0, stream=r, capacity=1 << 15))
    plan = abc.Plan(regs, wl[BATCH_REGIONS[0]]["seed"], mode="fast")
    s = torch.cuda.Stream(dev)
    best, shapes = plan.tune(s)
    with torch.cuda.stream(s):
        for _ in range(warmup):
            plan.run_graph(1, s)
        s.synchronize()
        plan.reset(s)
        before = [plan.counts(r, s) for r in range(len(regs))]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(s)
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(s)
            plan.run_graph(1, s)
            ev[k][1].record(s)
        r1.record(s)
        s.synchronize()
    counts = [plan.counts(r, s) for r in range(len(regs))]
    plan.close()
    acc = sum(c[0] for c in counts) - sum(b[0] for b in before)
    days = sum(c[1] for c in counts) - sum(b[1] for b in before)
    region_ms = r0.elapsed_time(r1)
    launch_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    nominal = sum(g["n_samples"] * (g["observed"].shape[1] - 1) for g in regs)
    return {"workload": "3 regions in one launch (" + ", ".join(
                "%s eps=%g" % (n, wl[n]["eps"]) for n in BATCH_REGIONS) + "), 2^22 prior samples each, fast mode, "
                "CUDA-graph replay, L2 flushed between steps",
            "value": acc / (region_ms * 1e-3), "unit": UNIT, "ms_per_step": region_ms / steps,
            "launch_ms_mean": launch_ms, "sims_days_per_s": nominal * steps / (region_ms * 1e-3),
            "simulated_days_per_step": days / steps, "accepted_per_step": acc / steps,
            "tuned_shape": best, "shapes_tried": shapes,
            "roofline": roofline(days / steps, launch_ms, sm_count, sm_max,
                                 samples_per_launch=sum(g["n_samples"] for g in regs))}


def bench_streamed(abc, torch, dev, flush, sm_count, sm_max, chunks=16):
    """Sixteen regions (P log-uniform in 1e6 .. 3e8, T uniform in 30 .. 180,
    own eps each) streamed in 2^24-sample chunks (2^20 per region per chunk),
    2^28 simulations in all, with the accepted samples accumulating in the
    plan's device-resident buffers; the chunks are one CUDA-graph replay."""
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        wl = json.load(f)
    names = sorted(k for k in wl if k.startswith("stream16_"))
    regs = [dict(observed=np.array(wl[nm]["observed"], dtype=np.int32), N_pop=wl[nm]["P"], eps=wl[nm]["eps"],
                 n_samples=wl[nm]["n_samples"], first_index=0, stream=r, capacity=1 << 16)
            for r, nm in enumerate(names)]
    plan = abc.Plan(regs, wl[names[0]]["seed"], mode="fast")
    s = torch.cuda.Stream(dev)
    best, _ = plan.tune(s)
    with torch.cuda.stream(s):
        plan.run_graph(chunks, s)          # warm-up replay (captures the graph)
        s.synchronize()
        plan.reset(s)
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        plan.run_graph(chunks, s)
        e1.record(s)
        s.synchronize()
    ms = e0.elapsed_time(e1)
    counts = [plan.counts(r, s) for r in range(len(regs))]
    plan.close()
    acc = sum(c[0] for c in counts)
    days = sum(c[1] for c in counts)
    nominal = chunks * sum(g["n_samples"] * (g["observed"].shape[1] - 1) for g in regs)
    return {"workload": "16 regions (P log-uniform 1e6..3e8, T uniform 30..180, own eps each), 2^28 prior samples "
                        "streamed in %d chunks of 2^24 in one CUDA-graph replay, fast mode" % chunks,
            "value": acc / (ms * 1e-3), "unit": UNIT, "ms_total": ms, "accepted": acc,
            "sims_days_per_s": nominal / (ms * 1e-3), "simulated_days": days, "tuned_shape": best,
            "roofline": roofline(days, ms, sm_count, sm_max,
                                 samples_per_launch=chunks * sum(g["n_samples"] for g in regs))}


def bench_config1(abc, torch, dev, reps=20, warmup=3):
    """Plain ABC on region_1e6_T49 (P = 1e6, T = 49): 65,536 prior samples,
    exact mode, eps at the 0.1 % distance quantile. One run is the whole
    pipeline through the public calls: every distance and prior draw, eps as
    the k-th smallest, k = ceil(0.001 n) = 66 (radix select on the device),
    then the samples at or below that eps from those distances (the same
    accepted set as a rejection launch at eps, without simulating again).
    Timed as one abc_sample_quantile call, and beside it as the three calls
    abc_distances, abc_kth_smallest and abc_select_below (each with its own
    synchronisation). The observed series comes from host memory in each
    call; eps and the accepted count are checked against the workload's own
    (written by the oracle)."""
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        w = json.load(f)["region_1e6_T49"]
    obs, P, T, n, seed = np.array(w["observed"], dtype=np.int32), w["P"], w["T"], w["n_samples"], w["seed"]
    k = int(np.ceil(0.001 * n))
    cap = 1024
    outs = (torch.empty((cap, 8), dtype=torch.float32, device=dev), torch.empty((cap,), dtype=torch.float64, device=dev),
            torch.empty((cap,), dtype=torch.int64, device=dev))
    dbuf = torch.empty((n,), dtype=torch.float64, device=dev)
    tbuf = torch.empty((n, 8), dtype=torch.float32, device=dev)
    stage = {"distances": [], "kth_smallest": [], "select": []}
    walls, walls3, eps, n_acc, eps3, n_acc3 = [], [], None, None, None, None
    for rep in range(warmup + reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, n_acc, eps = abc.abc_sample_quantile(obs, P, n, k, seed, mode="exact", out=outs)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        d, th = abc.abc_distances(obs, P, n, seed, mode="exact", want_theta=True, out=(dbuf, tbuf))
        ev[1].record()
        eps3 = abc.abc_kth_smallest(d, k)
        ev[2].record()
        _, _, _, n_acc3 = abc.abc_select_below(d, eps3, theta=th, out=outs)
        ev[3].record()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if rep >= warmup:
            walls.append(t1 - t0)
            walls3.append(t2 - t1)
            for j, key in enumerate(stage):
                stage[key].append(ev[j].elapsed_time(ev[j + 1]))
    ms = float(np.median(walls)) * 1e3
    ms3 = float(np.median(walls3)) * 1e3
    out = {"workload": "region_1e6_T49: P=1e6, T=49, %d prior samples, exact mode, eps = %d-th smallest distance "
                       "(0.1 %% quantile)" % (n, k),
           "accepted": int(n_acc), "eps": eps, "eps_equals_workload": bool(eps == w["eps"]),
           "ms_per_run": ms, "accepted_per_s": n_acc / (ms * 1e-3),
           "sims_days_per_s": n * T / (ms * 1e-3),
           "three_calls": {"ms_per_run": ms3, "same_eps_and_count": bool(eps3 == eps and n_acc3 == n_acc),
                           "ms_by_stage": {key: float(np.median(v)) for key, v in stage.items()}},
           "runs": reps}
    return out


def cpu_baseline_config1():
    """The oracle on the same pipeline on the host cores: every distance of
    region_1e6_T49's 65,536 samples (all cores), eps as the 66-th smallest, and
    the accepted samples at that eps."""
    import oracle
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        w = json.load(f)["region_1e6_T49"]
    obs, n = np.array(w["observed"], dtype=np.int32), w["n_samples"]
    k = int(np.ceil(0.001 * n))
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    d = oracle.abc(obs, w["P"], 0.0, n, w["seed"], want_all=True, capacity=1, n_threads=cores)["dist_all"]
    eps = float(np.partition(d, k - 1)[k - 1])
    acc = int(np.count_nonzero(d <= eps))
    dt = time.perf_counter() - t0
    return {"value": acc / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt, "accepted": acc,
            "sample": "the whole workload (%d samples), distances on %d threads" % (n, cores)}


def bench_exact(abc, torch, w, dev, flush, fast_days_per_s, steps=5, warmup=3, n=1 << 22):
    """The headline workload in exact mode (the project's own FP32 series, no
    FMA contraction: bit-exact against the CPU oracle), 2^22 samples per
    launch on fresh indices, L2 flushed between launches; the cost of exactness
    as simulated days per second against fast mode."""
    obs_dev = abc.Observed(w["observed"], w["P"])
    cap = 1 << 14
    outs = (torch.empty((cap, 8), dtype=torch.float32, device=dev), torch.empty((cap,), dtype=torch.float64, device=dev),
            torch.empty((cap,), dtype=torch.int64, device=dev))
    cnt = torch.zeros((warmup + steps, 4), dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream(dev)
    first = 1 << 40
    for k in range(warmup):
        abc.abc_sample_async(obs_dev, w["eps"], n, w["seed"], outs, cnt[k], mode="exact", first_index=first + k * n,
                             cuda_stream=s)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(s)
        abc.abc_sample_async(obs_dev, w["eps"], n, w["seed"], outs, cnt[warmup + k], mode="exact",
                             first_index=first + (warmup + k) * n, cuda_stream=s)
        ev[k][1].record(s)
    torch.cuda.synchronize()
    obs_dev.close()
    ms = float(sum(a.elapsed_time(b) for a, b in ev))
    c = cnt[warmup:].cpu().numpy()
    acc, days = int(c[:, 0].sum()), int(c[:, 2].sum())
    dps = days / (ms * 1e-3)
    return {"workload": "region_6e7_T100 in exact mode, %d prior samples per launch, %d launches, eps=%g" % (
                n, steps, w["eps"]),
            "accepted_per_s": acc / (ms * 1e-3), "unit": UNIT, "ms_per_launch": ms / steps,
            "simulated_days_per_s": dps, "fast_simulated_days_per_s": fast_days_per_s,
            "exact_over_fast": dps / fast_days_per_s}


def bench_projection(abc, torch, w, B=8192, T=120, reps=10):
    """Posterior-predictive projection (Sec. 5: accepted samples simulated 120
    days forward, 5th-95th percentile bands): B accepted samples of the
    headline workload re-simulated from its initial condition for T days,
    with bands at the 5, 50 and 95 % quantiles of every (day, compartment)."""
    th, _, idx, n = abc.abc_sample(w["observed"], w["P"], w["eps"], 6 << 24, w["seed"], first_index=1 << 36,
                                   capacity=1 << 15)
    m = min(B, th.shape[0])
    th, idx = th[:m].contiguous(), idx[:m].contiguous()
    s = torch.cuda.Stream()

    def timed(fn):
        with torch.cuda.stream(s):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
        s.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: abc.abc_project(th, idx, w["observed"][:, 0], T, w["P"], w["seed"], cuda_stream=s))
    ms_sim = timed(lambda: abc.abc_simulate(th, idx, w["observed"][:, 0], T, w["P"], w["seed"], mode="fast",
                                            cuda_stream=s))
    # one thread per trajectory: 8192 trajectories are 1.7 warps per SM, so the
    # call is latency-bound by its size (Sec. 5 projects 100 samples)
    return {"workload": "%d accepted samples of region_6e7_T100 simulated %d days from its initial condition, "
                        "bands at the 5, 50, 95 %% quantiles, fast mode" % (m, T),
            "ms_per_projection": ms, "ms_trajectories": ms_sim, "ms_bands": ms - ms_sim,
            "trajectories_per_s": m / (ms * 1e-3), "simulated_days_per_s": m * T / (ms * 1e-3)}


def bench_pmc(abc, torch, w, prior_value, rounds=4, factor=0.7):
    """Population Monte Carlo ABC (Beaumont et al. 2009, the SMC-ABC of
    Sec. 2.2) on the headline region, 4 rounds of 4096 particles ending at the
    headline eps, proposals in batches of 2^22."""
    eps0 = w["eps"] / factor ** (rounds - 1)
    info, th, wt, dist = abc.abc_pmc_run(w["observed"], w["P"], eps0, rounds=rounds, n_particles=4096,
                                         batch=1 << 22, max_batches=64, eps_factor=factor, seed=w["seed"] + 5,
                                         capacity=1 << 17, mode="fast")
    last = info[-1]
    ms = last["ms"]
    eff = ess(wt.cpu().numpy())
    return {"workload": "population Monte Carlo ABC, region_6e7_T100, %d rounds of 4096 particles, eps0=%g, "
                        "factor %g, final eps=%g (the headline eps), batches of 2^22" % (rounds, eps0, factor, w["eps"]),
            "final_round_accepted_per_s": last["n_accepted"] / (ms * 1e-3),
            "final_round_effective_accepted_per_s": eff / (ms * 1e-3),
            "final_round_simulations": last["n_sims"], "final_round_ess_fraction": last["ess_fraction"],
            "prior_accepted_per_s_same_eps": prior_value,
            "gain_effective_vs_prior": eff / (ms * 1e-3) / prior_value,
            "all_rounds_seconds": sum(r["ms"] for r in info) * 1e-3}


def bench_literal(abc, torch, w, dev, flush, fast_days_per_s, steps=5, warmup=3, n=1 << 24):
    """The literal-variance model variant (transition draws with standard
    deviation h^(1/4)) on the headline workload and eps, fast mode."""
    obs_dev = abc.Observed(w["observed"], w["P"])
    cap = 1 << 20
    outs = (torch.empty((cap, 8), dtype=torch.float32, device=dev), torch.empty((cap,), dtype=torch.float64, device=dev),
            torch.empty((cap,), dtype=torch.int64, device=dev))
    cnt = torch.zeros((warmup + steps, 4), dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream(dev)
    first = 1 << 41
    for k in range(warmup):
        abc.abc_sample_async(obs_dev, w["eps"], n, w["seed"], outs, cnt[k], mode="fast_literal",
                             first_index=first + k * n, cuda_stream=s)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(s)
        abc.abc_sample_async(obs_dev, w["eps"], n, w["seed"], outs, cnt[warmup + k], mode="fast_literal",
                             first_index=first + (warmup + k) * n, cuda_stream=s)
        ev[k][1].record(s)
    torch.cuda.synchronize()
    obs_dev.close()
    ms = float(sum(a.elapsed_time(b) for a, b in ev))
    c = cnt[warmup:].cpu().numpy()
    acc, days = int(c[:, 0].sum()), int(c[:, 2].sum())
    return {"workload": "region_6e7_T100, literal-variance model, %d prior samples per launch, %d launches, eps=%g"
                        % (n, steps, w["eps"]),
            "accepted_per_s": acc / (ms * 1e-3), "unit": UNIT, "ms_per_launch": ms / steps,
            "simulated_days_per_s": days / (ms * 1e-3), "standard_model_simulated_days_per_s": fast_days_per_s,
            "acceptance": acc / (steps * n)}


def ess(w):
    w = np.asarray(w, dtype=np.float64)
    return float(w.sum() ** 2 / (w ** 2).sum()) if len(w) else 0.0


# learned proposals: flow base broadened by 1.25, training weights w^0.8
LEARNED_TAU, LEARNED_POWER = 1.25, 0.8


def bench_learned_stream(abc, torch, prior_stream=None):
    """Sixteen regions (the streamed leg's), one flow proposal per region:
    16 rounds, each one batched launch of 2^20 simulations per region (2^24
    per chunk, 2^28 in all); eps shrinks by 0.7 per round to each region's
    final eps over the first 4 rounds, then stays there while the samples
    accepted at the final eps pool in device buffers with their importance
    weights; the 16 flows (3 x 256, BF16) train together after every round
    on batches of 2048 rows each,
    a region falling back to the prior whenever its ESS fraction drops below
    10 %."""
    with open(os.path.join(ROOT, "tests", "golden", "workloads.json")) as f:
        wl = json.load(f)
    names = sorted(k for k in wl if k.startswith("stream16_"))
    regs = [dict(observed=np.array(wl[nm]["observed"], dtype=np.int32), N_pop=wl[nm]["P"], eps=wl[nm]["eps"],
                 pool=1 << 21) for nm in names]
    rounds, shrink, n = 16, 4, 1 << 20
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info, res = abc.abc_smc_run_regions(regs, rounds=rounds, shrink_rounds=shrink, sims_per_round=n, eps_factor=0.7,
                                        flow_blocks=3, flow_hidden=256, train_steps=500, train_steps_warm=100,
                                        train_batch=2048, train_lr=1e-3, seed=wl[names[0]]["seed"] + 29,
                                        capacity=1 << 20, mode="fast", proposal_scale=LEARNED_TAU,
                                        train_weight_power=LEARNED_POWER, fallback="ess")
    wall = time.perf_counter() - t0
    pooled = sum(r[3] for r in res)
    eff = sum(ess(r[1].cpu().numpy()) for r in res)
    dev_s = sum(info[r][0]["ms_propose"] + info[r][0]["ms_simulate"] + info[r][0]["ms_train"] for r in range(rounds))
    out = {"workload": "16 regions (P log-uniform 1e6..3e8, T uniform 30..180, own final eps each), one flow "
                       "proposal per region (3 x 256 BF16), %d rounds x 2^20 simulations per region (2^24 per "
                       "chunk, 2^28 in all), eps x0.7 per round over the first %d rounds, prior fallback when a "
                       "region's ESS fraction drops below 10 %%, fast mode" % (rounds, shrink),
           "seconds": wall, "device_seconds_by_round_events": dev_s * 1e-3,
           "propose_seconds": sum(info[r][0]["ms_propose"] for r in range(rounds)) * 1e-3,
           "simulate_seconds": sum(info[r][0]["ms_simulate"] for r in range(rounds)) * 1e-3,
           "weights_and_train_seconds": sum(info[r][0]["ms_train"] for r in range(rounds)) * 1e-3,
           "pooled_accepted_at_final_eps": pooled, "pooled_effective": eff,
           "accepted_per_s": pooled / wall, "effective_accepted_per_s": eff / wall,
           "flow_rounds": int(sum(info[r][g]["proposal"] for r in range(rounds) for g in range(len(regs)))),
           "fallback_rounds": int(sum(1 - info[r][g]["proposal"] for r in range(1, rounds) for g in range(len(regs)))),
           "min_ess_fraction": min(info[r][g]["ess_fraction"] for r in range(rounds) for g in range(len(regs))
                                   if info[r][g]["n_accepted"] > 0)}
    if prior_stream:
        out["prior_stream_accepted_per_s"] = prior_stream["value"]
        out["gain_effective_vs_prior_stream"] = out["effective_accepted_per_s"] / prior_stream["value"]
    return out


def bench_learned(abc, torch, w, prior_value, peaks, sm_count, sm_max, reps=5, verbose=False):
    """Sequential ABC with the learned flow proposal on the P = 6e7, T = 100
    region: 5 rounds of 2^22 simulations, eps shrinking by 0.7 per round to the
    headline eps, flow of 3 MADE blocks x 256 hidden units (BF16 weights, FP32
    accumulation), proposals from the flow broadened by LEARNED_TAU. Compared
    with plain prior ABC at the same (final) eps.

    The headline figure is the whole run: effective samples accepted at the
    final eps (accepted x ESS fraction of the final round, the only round at
    that eps) per second of the whole abc_smc_run call, all five rounds with
    their proposals, simulations, weights and training. The final round alone
    (proposals and simulations) is reported beside it. The flow's training is
    stochastic, so `reps` independent runs (own seeds) are made; medians are
    reported, with every run listed."""
    rounds, n, factor = 5, 1 << 22, 0.7
    eps0 = w["eps"] / factor ** (rounds - 1)
    runs = []
    for rep in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, th, wt, dist = abc.abc_smc_run(w["observed"], w["P"], eps0, rounds=rounds, sims_per_round=n,
                                             eps_factor=factor, flow_blocks=3, flow_hidden=256, train_steps=500,
                                             train_batch=4096, train_lr=1e-3, seed=w["seed"] + 17 + 1000 * rep,
                                             capacity=n, mode="fast", proposal_scale=LEARNED_TAU,
                                             train_weight_power=LEARNED_POWER)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        last = info[-1]
        ms = last["ms_propose"] + last["ms_simulate"]
        eff = last["n_accepted"] * last["ess_fraction"]
        run = {"seed": w["seed"] + 17 + 1000 * rep,
               "final_round_proposal": "flow" if last["proposal"] == 1 else "prior (fallback)",
               "whole_run_seconds": wall,
               "whole_run_effective_accepted_per_s": eff / wall,
               "final_round_accepted_per_s": last["n_accepted"] / (ms * 1e-3),
               "final_round_effective_accepted_per_s": eff / (ms * 1e-3),
               "final_round_acceptance": last["n_accepted"] / n,
               "final_round_ess_fraction": last["ess_fraction"],
               "device_seconds": sum(r["ms_propose"] + r["ms_simulate"] + r["ms_train"] for r in info) * 1e-3,
               "ms_propose": last["ms_propose"], "ms_simulate": last["ms_simulate"],
               "final_round_simulated_days": last["simulated_days"]}
        if verbose:
            run["rounds"] = [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()} for r in info]
        runs.append(run)
    med = lambda key: float(np.median([r[key] for r in runs]))
    flow_runs = [r for r in runs if r["final_round_proposal"] == "flow"]
    out = {"workload": "sequential ABC, region_6e7_T100, %d rounds x 2^22, eps x%g per round to the headline eps, "
                       "flow 3 x 256 BF16, %d runs (medians)" % (rounds, factor, reps),
           "whole_run_effective_accepted_per_s": med("whole_run_effective_accepted_per_s"),
           "whole_run_gain_effective_vs_prior": med("whole_run_effective_accepted_per_s") / prior_value,
           "whole_run_seconds": med("whole_run_seconds"),
           "final_round_accepted_per_s": med("final_round_accepted_per_s"),
           "final_round_effective_accepted_per_s": med("final_round_effective_accepted_per_s"),
           "final_round_gain_effective_vs_prior": med("final_round_effective_accepted_per_s") / prior_value,
           "final_round_acceptance": med("final_round_acceptance"),
           "runs_ending_on_prior_fallback": reps - len(flow_runs),
           "prior_accepted_per_s_same_eps": prior_value,
           "whole_run_effective_per_s_by_run": [round(r["whole_run_effective_accepted_per_s"], -3) for r in runs],
           "runs": runs}
    if flow_runs:
        # the final round's simulations of flow proposals (batched kernel with a
        # proposal buffer) against the same ALU roofline as the headline
        sims = sorted(flow_runs, key=lambda r: r["final_round_simulated_days"] / r["ms_simulate"])
        mid = sims[len(sims) // 2]
        out["simulate_roofline"] = roofline(mid["final_round_simulated_days"], mid["ms_simulate"], sm_count, sm_max,
                                            samples_per_launch=n)
        ms_prop = float(np.median([r["ms_propose"] for r in flow_runs]))
        # algorithmic work per proposal: every hidden unit once per block (the
        # sampler adds each unit's contribution when its inputs are final), the
        # masked MADE's nonzero multiply-adds: unit l of degree d = l mod 7 + 1
        # reads d inputs and feeds 8 - d means and 8 - d log-scales
        H, blocks = 256, 3
        macs = sum(16 - (l % 7 + 1) for l in range(H))
        n_flow = int(0.9 * n)
        flops = 2 * macs * blocks * n_flow
        measured = "bf16_tflops" in (peaks or {})
        peak = peaks["bf16_tflops"] if measured else 1900.0
        achieved = flops / (ms_prop * 1e-3) / 1e12
        out["sampler_roofline"] = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                   "frac": achieved / peak, "traffic": None, "ms_propose": ms_prop,
                                   "peak_source": "measured" if measured else "fallback",
                                   "basis": "%d FLOP per flow proposal (masked MADE nonzero multiply-adds), %d flow "
                                            "proposals per round; peak = %s"
                                            % (flops // n_flow, n_flow,
                                               "the measured cuBLAS bf16 burst" if measured
                                               else "the fallback bf16 burst figure, 1.9 PFLOP/s (no measured peaks file)")}
    return out


def summary(line):
    """The workloads' figures in one short object, last on the line."""
    def r4(x):
        return float("%.4g" % x) if isinstance(x, float) else x
    out = {"c2_headline": {"accepted_per_s": r4(line["value"]), "frac": r4(line["roofline"]["frac"]),
                           "days_only_frac": r4(line["roofline"]["days_only_frac"]),
                           "e2e_accepted_per_s": r4((line.get("e2e") or {}).get("value"))}}
    c1 = line.get("config1")
    if c1:
        out["c1_exact_quantile"] = {"accepted": c1["accepted"], "ms_per_run": r4(c1["ms_per_run"]),
                                    "accepted_per_s": r4(c1["accepted_per_s"]), "eps_ok": c1["eps_equals_workload"],
                                    "three_calls_ms": r4(c1["three_calls"]["ms_per_run"]),
                                    "oracle_s": r4((c1.get("cpu_baseline") or {}).get("seconds"))}
    b = line.get("batched_regions")
    if b:
        out["c3_batched"] = {"accepted_per_s": r4(b["value"]), "frac": r4(b["roofline"]["frac"]),
                             "days_only_frac": r4(b["roofline"]["days_only_frac"])}
    lp = line.get("learned_proposal")
    if lp:
        out["c4_learned"] = {"whole_run_gain": r4(lp["whole_run_gain_effective_vs_prior"]),
                             "whole_run_effective_per_s": r4(lp["whole_run_effective_accepted_per_s"]),
                             "final_round_gain": r4(lp["final_round_gain_effective_vs_prior"]),
                             "whole_run_s": r4(lp["whole_run_seconds"])}
    st = line.get("streamed_regions")
    if st:
        out["c5_prior_stream"] = {"accepted_per_s": r4(st["value"]), "frac": r4(st["roofline"]["frac"]),
                                  "days_only_frac": r4(st["roofline"]["days_only_frac"])}
    ls = line.get("learned_stream")
    if ls:
        out["c5_learned_stream"] = {"effective_per_s": r4(ls["effective_accepted_per_s"]),
                                    "gain_vs_prior_stream": r4(ls.get("gain_effective_vs_prior_stream", float("nan"))),
                                    "seconds": r4(ls["seconds"])}
    return out


def oracle_sample(w, n, first_index, threads=0):
    """The CPU oracle (exact arithmetic) on n samples of the workload."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.abc(w["observed"], w["P"], w["eps"], n, w["seed"], first_index=first_index,
                   capacity=max(64, n // 100), n_threads=threads)
    return time.perf_counter() - t0, r["n_accepted"]


def cpu_baseline(w, n=1 << 20):
    cores = os.cpu_count() or 1
    dt, acc = oracle_sample(w, n, 0, cores)
    return {"value": acc / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sims_days_per_s": n * w["T"] / dt, "accepted": acc, "seconds": dt,
            "sample": "%d prior samples (indices 0..%d) of the same workload and eps, C oracle, %d threads" % (
                n, n - 1, cores)}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = load_workload()
    n = 1 << 18
    for s in range(args.warmup):
        oracle_sample(w, n, s * n)
    tot, acc = 0.0, 0
    for s in range(args.steps):
        dt, a = oracle_sample(w, n, (args.warmup + s) * n)
        tot += dt
        acc += a
    cores = os.cpu_count() or 1
    value = acc / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": describe(w) + "; reference arm = the C oracle "
                                                            "(exact-mode arithmetic) on the host cores",
                                            "samples_per_step": n, "parallelism": "host threads"},
            "sims_days_per_s": n * args.steps * w["T"] / tot,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d prior samples per step of the same workload and eps" % n},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-streamed", action="store_true")
    ap.add_argument("--no-learned-stream", action="store_true")
    ap.add_argument("--no-exact", action="store_true")
    ap.add_argument("--no-next", action="store_true", help="skip the projection, PMC and literal-model legs")
    ap.add_argument("--no-config1", action="store_true")
    ap.add_argument("--verbose", action="store_true", help="per-round detail of the learned runs")
    ap.add_argument("--leg", default="all", choices=["all", "headline", "batched", "learned", "streamed",
                                                     "learned_stream", "exact", "projection", "pmc", "literal",
                                                     "config1"],
                    help="run one leg only (profiling); 'all' is the benchmark")
    ap.add_argument("--samples", type=int, default=0,
                    help="samples per launch (profiling runs on a smaller case; not a benchmark value)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2012_14332_gb300 as abc
    from paper_2012_14332_gb300 import build as abc_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(abc_build.LIB):
        abc_build.build()
    if dist is not None:
        dist.barrier()
    abc.load()

    w = load_workload()
    if args.samples:
        w["n_samples"] = args.samples
    obs, P, T, n, seed, eps = w["observed"], w["P"], w["T"], w["n_samples"], w["seed"], w["eps"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cap = 1 << 16
    outs = (torch.empty((cap, 8), dtype=torch.float32, device=dev), torch.empty((cap,), dtype=torch.float64, device=dev),
            torch.empty((cap,), dtype=torch.int64, device=dev))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def first_index(step):
        return (step * world + rank) * n

    # the observed series is uploaded once; each step enqueues one launch whose
    # counters (accepted, processed, simulated days) stay on the device until
    # the timed region ends, so steps run back to back with no host round trip
    obs_dev = abc.Observed(obs, P)
    counters = torch.zeros((args.warmup + args.steps, 4), dtype=torch.int64, device=dev)

    def step(s):
        abc.abc_sample_async(obs_dev, eps, n, seed, outs, counters[s], mode=w["mode"], first_index=first_index(s),
                             cuda_stream=stream)

    if args.leg in ("batched", "learned", "streamed", "learned_stream", "exact", "projection", "pmc", "literal",
                    "config1"):
        props = torch.cuda.get_device_properties(dev)
        peaks = measured_peaks() or {}
        if args.leg == "config1":
            out = bench_config1(abc, torch, dev)
        elif args.leg == "batched":
            out = bench_batched(abc, torch, args.steps, args.warmup, dev, flush, props.multi_processor_count,
                                peaks.get("sm_max_mhz", 2070.0))
        elif args.leg == "streamed":
            out = bench_streamed(abc, torch, dev, flush, props.multi_processor_count, peaks.get("sm_max_mhz", 2070.0))
        elif args.leg == "learned_stream":
            out = bench_learned_stream(abc, torch)
        elif args.leg == "exact":
            out = bench_exact(abc, torch, w, dev, flush, float("nan"))
        elif args.leg == "projection":
            out = bench_projection(abc, torch, w)
        elif args.leg == "pmc":
            out = bench_pmc(abc, torch, w, float("nan"))
        elif args.leg == "literal":
            out = bench_literal(abc, torch, w, dev, flush, float("nan"))
        else:
            out = bench_learned(abc, torch, w, float("nan"), peaks, props.multi_processor_count,
                                peaks.get("sm_max_mhz", 2070.0), verbose=args.verbose)
        print(json.dumps({"leg": args.leg, **out}), flush=True)
        return
    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    region0, region1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    region0.record(stream)
    for s in range(args.steps):
        flush.fill_(s & 0xFF)                       # evict L2 between steps
        starts[s].record(stream)
        step(args.warmup + s)
        ends[s].record(stream)
    region1.record(stream)
    torch.cuda.synchronize()
    cnt = counters[args.warmup:].cpu().numpy()
    if (cnt[:, 0] > cap).any():
        raise RuntimeError("more accepted samples in a step than the output capacity %d" % cap)
    accepted = int(cnt[:, 0].sum())
    sim_days = [int(cnt[:, 2].sum())]
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    region_ms = region0.elapsed_time(region1)
    launch_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    t_region = torch.tensor([region_ms, float(accepted)], dtype=torch.float64, device=dev)
    if dist is not None:
        tmax = t_region.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t_region.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        region_ms, accepted = float(tmax[0]), int(tsum[1])
    ms_per_step = region_ms / args.steps
    sims_per_step = n * world
    value = accepted / (region_ms * 1e-3)

    # end to end through the public call with host buffers: observed series from
    # pinned host memory inside the call, accepted samples copied back to pinned
    # host memory inside the timed region
    host_theta = torch.empty((cap, 8), dtype=torch.float32, pin_memory=True)
    host_dist = torch.empty((cap,), dtype=torch.float64, pin_memory=True)
    host_idx = torch.empty((cap,), dtype=torch.int64, pin_memory=True)
    obs_pinned = torch.from_numpy(obs).pin_memory().numpy()
    e2e_steps = 0 if args.no_e2e else max(3, args.steps // 2)
    d2h, e2e_accepted = 0, 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(e2e_steps):
        th, di, ix, a = abc.abc_sample(obs_pinned, P, eps, n, seed, mode=w["mode"],
                                       first_index=first_index(args.warmup + args.steps + s), capacity=cap, out=outs)
        m = th.shape[0]
        e2e_accepted += a
        host_theta[:m].copy_(th, non_blocking=True)
        host_dist[:m].copy_(di, non_blocking=True)
        host_idx[:m].copy_(ix, non_blocking=True)
        d2h += 8 + m * (32 + 8 + 8)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    e2e_n = torch.tensor([float(e2e_accepted)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e2e_n, op=dist.ReduceOp.SUM)
    e2e_s, e2e_accepted = float(e2e_t[0]), int(e2e_n[0])

    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        peaks = measured_peaks() or {}
        sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
        rf = roofline(sim_days[0] / args.steps, float(np.mean(launch_ms)), props.multi_processor_count, sm_max,
                      traffic=REJECT_TRAFFIC_BYTES if w["n_samples"] == 1 << 24 else None, samples_per_launch=n)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe(w), "samples_per_step": sims_per_step,
                       "parallelism": "dp%d" % world, "l2": "flushed between steps (256 MiB write)",
                       "timed_call": "abc_sample_async: observed series resident on the device, one launch per step, "
                                     "counters read after the timed region",
                       "eps": eps, "seed": seed},
            "sims_days_per_s": sims_per_step * T / (ms_per_step * 1e-3),
            "simulated_days_per_step": sim_days[0] / args.steps,
            "early_rejection": "samples whose running distance^2 exceeds eps^2 stop early; sims_days_per_s counts "
                               "n_samples * T, simulated_days_per_step the days actually run",
            "accepted_per_step": accepted / args.steps,
            "acceptance": accepted / (args.steps * sims_per_step),
            "launch_ms_mean": float(np.mean(launch_ms)),
            "e2e": ({"value": e2e_accepted / e2e_s, "unit": UNIT, "ms_per_step": e2e_s / e2e_steps * 1e3,
                     "h2d_bytes_per_step": 16 * (T + 1), "d2h_bytes_per_step": int(d2h / e2e_steps)}
                    if e2e_steps else None),
            "gpu_launches": args.steps,
            "roofline": rf,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        if args.leg == "headline":
            args.no_learned = args.no_batched = args.no_streamed = args.no_learned_stream = args.no_exact = True
            args.no_next = args.no_config1 = True
        if not args.no_config1 and world == 1:
            line["config1"] = bench_config1(abc, torch, dev)
            if not args.no_cpu_baseline:
                line["config1"]["cpu_baseline"] = cpu_baseline_config1()
        if not args.no_exact and world == 1:
            line["exact_mode"] = bench_exact(abc, torch, w, dev, flush, sim_days[0] / (float(np.sum(launch_ms)) * 1e-3))
        if not args.no_learned and world == 1:
            line["learned_proposal"] = bench_learned(abc, torch, w, value, peaks, props.multi_processor_count, sm_max,
                                                     verbose=args.verbose)
        if not args.no_batched and world == 1:
            line["batched_regions"] = bench_batched(abc, torch, args.steps, args.warmup, dev, flush,
                                                    props.multi_processor_count, sm_max)
        if not args.no_streamed and world == 1:
            line["streamed_regions"] = bench_streamed(abc, torch, dev, flush, props.multi_processor_count, sm_max)
        if not args.no_learned_stream and world == 1:
            line["learned_stream"] = bench_learned_stream(abc, torch, line.get("streamed_regions"))
        if not args.no_next and world == 1:
            fast_dps = sim_days[0] / (float(np.sum(launch_ms)) * 1e-3)
            line["projection"] = bench_projection(abc, torch, w)
            line["pmc"] = bench_pmc(abc, torch, w, value)
            line["literal_model"] = bench_literal(abc, torch, w, dev, flush, fast_dps)
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
