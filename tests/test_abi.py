"""The C-ABI library without a GPU: it builds, loads, exports every entry
point that include/abc_gb300.h declares, and rejects invalid arguments before
any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "abc_gb300.h")


@pytest.fixture(scope="module")
def L():
    from paper_2012_14332_gb300 import build, load
    build.build()
    return load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(abc_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("abc_sample", "abc_distances", "abc_simulate", "abc_step", "abc_kth_smallest", "abc_strerror",
                 "abc_last_error", "abc_version"):
        assert must in names, names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_binding_names_match_header():
    import paper_2012_14332_gb300.binding as b
    for name in declared_functions():
        if name not in ("abc_last_error",):
            assert hasattr(b, name), name


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and
    field offsets (gcc on the header itself), so no field is dropped,
    reordered or mistyped on either side of the boundary."""
    import shutil
    import subprocess
    import paper_2012_14332_gb300.binding as b
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"abc_prior_box": b.AbcPriorBox, "abc_region": b.AbcRegion, "abc_launch_shape": b.AbcLaunchShape,
             "abc_smc_config": b.AbcSmcConfig, "abc_smc_round": b.AbcSmcRound, "abc_smc_region": b.AbcSmcRegion,
             "abc_smc_stream_config": b.AbcSmcStreamConfig, "abc_pmc_config": b.AbcPmcConfig,
             "abc_pmc_round": b.AbcPmcRound}
    src = open(HEADER).read()
    lines, want = [], []
    for cname, cls in pairs.items():
        assert re.search(r"\}\s*%s\s*;" % cname, src), cname
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        want.append(ctypes.sizeof(cls))
        for f in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f[0]))
            want.append(getattr(cls, f[0]).offset)
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "abc_gb300.h"\nint main(void) {\n%s\nreturn 0;\n}\n'
                    % "\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.dirname(HEADER), "-o", str(exe), str(prog)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == want


def test_strerror_and_version(L):
    from paper_2012_14332_gb300 import binding as b
    for st in range(6):
        assert L.abc_strerror(st)
    assert L.abc_strerror(99) == b"unknown status"
    assert L.abc_version() >= 100


def _call_sample(L, **kw):
    from paper_2012_14332_gb300.binding import prior_box
    T = kw.get("T", 10)
    obs = kw.get("observed", np.zeros((3, T + 1), dtype=np.int32))
    obs = np.ascontiguousarray(obs, dtype=np.int32)
    box = kw.get("box", prior_box())
    n = ctypes.c_uint64(0)
    bogus = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    return L.abc_sample(ctypes.byref(box) if box is not None else None,
                        obs.ctypes.data_as(ctypes.c_void_p) if kw.get("obs_null") is None else None,
                        T, kw.get("P", 1000), kw.get("eps", 1.0), kw.get("n", 10), 1, kw.get("stream", 0),
                        kw.get("mode", 1), kw.get("first", 0), bogus, bogus, bogus, kw.get("cap", 4),
                        ctypes.byref(n) if not kw.get("nacc_null") else None, None)


@pytest.mark.parametrize("kw,fragment", [
    (dict(T=0), "T = 0"),
    (dict(T=4097), "T = 4097"),
    (dict(P=0), "N_pop"),
    (dict(P=2**31), "N_pop"),
    (dict(eps=-1.0), "eps"),
    (dict(eps=float("nan")), "eps"),
    (dict(mode=7), "mode"),
    (dict(stream=2**30), "stream"),
    (dict(first=2**64 - 5), "overflows"),
    (dict(box=None), "prior"),
    (dict(obs_null=True), "observed"),
    (dict(nacc_null=True), "n_accepted"),
])
def test_sample_rejects_invalid_arguments(L, kw, fragment):
    from paper_2012_14332_gb300.binding import ABC_ERR_INVALID_ARG
    assert _call_sample(L, **kw) == ABC_ERR_INVALID_ARG
    assert fragment in L.abc_last_error().decode()


def test_sample_rejects_bad_prior_and_observed(L):
    from paper_2012_14332_gb300.binding import ABC_ERR_INVALID_ARG, prior_box
    hi = np.array([1, 100, 2, 1, 1, 1, 1, 2], dtype=np.float32)
    lo = hi.copy()
    lo[3] = 5.0
    assert _call_sample(L, box=prior_box(lo, hi)) == ABC_ERR_INVALID_ARG
    lo = np.zeros(8, dtype=np.float32)
    lo[0] = np.inf
    assert _call_sample(L, box=prior_box(lo, hi)) == ABC_ERR_INVALID_ARG
    obs = np.zeros((3, 11), dtype=np.int32)
    obs[1, 5] = -1
    assert _call_sample(L, observed=obs) == ABC_ERR_INVALID_ARG
    obs = np.zeros((3, 11), dtype=np.int32)
    obs[:, 0] = [600, 300, 200]   # A0 + R0 + D0 > P = 1000
    assert _call_sample(L, observed=obs) == ABC_ERR_INVALID_ARG
    assert "exceeds" in L.abc_last_error().decode()


def test_other_entry_points_validate(L):
    from paper_2012_14332_gb300.binding import ABC_ERR_INVALID_ARG
    z = ctypes.c_void_p(16)
    init = np.array([10, 0, 0], dtype=np.int32)
    ip = init.ctypes.data_as(ctypes.c_void_p)
    assert L.abc_simulate(z, z, 4, ip, 0, 1000, 1, 0, 0, z, None) == ABC_ERR_INVALID_ARG
    assert L.abc_simulate(None, z, 4, ip, 10, 1000, 1, 0, 0, z, None) == ABC_ERR_INVALID_ARG
    big = np.array([900, 200, 0], dtype=np.int32)
    assert L.abc_simulate(z, z, 4, big.ctypes.data_as(ctypes.c_void_p), 10, 1000, 1, 0, 0, z, None) \
        == ABC_ERR_INVALID_ARG
    assert L.abc_step(z, z, z, None, 4, 1000, 1, 0, 0, z, None, None) == ABC_ERR_INVALID_ARG
    assert L.abc_step(z, z, z, z, 4, 0, 1, 0, 0, z, None, None) == ABC_ERR_INVALID_ARG
    out = ctypes.c_double()
    assert L.abc_kth_smallest(z, 10, 0, ctypes.byref(out), None) == ABC_ERR_INVALID_ARG
    assert L.abc_kth_smallest(z, 10, 11, ctypes.byref(out), None) == ABC_ERR_INVALID_ARG
    m = ctypes.c_uint64(5)
    assert L.abc_select_below(z, None, 10, -1.0, 0, None, z, z, 4, ctypes.byref(m), None) == ABC_ERR_INVALID_ARG
    assert m.value == 0
    assert L.abc_select_below(z, None, 10, float("nan"), 0, None, z, z, 4, ctypes.byref(m), None) \
        == ABC_ERR_INVALID_ARG
    assert L.abc_select_below(None, None, 10, 1.0, 0, None, z, z, 4, ctypes.byref(m), None) == ABC_ERR_INVALID_ARG
    assert L.abc_select_below(z, z, 10, 1.0, 0, None, z, z, 4, ctypes.byref(m), None) == ABC_ERR_INVALID_ARG
    assert L.abc_select_below(z, None, 10, 1.0, 0, None, z, z, 4, None, None) == ABC_ERR_INVALID_ARG
    assert L.abc_select_below(z, None, 10, 1.0, ~0 & (2**64 - 1), None, z, z, 4, ctypes.byref(m), None) \
        == ABC_ERR_INVALID_ARG
    assert L.abc_select_below(None, None, 0, 1.0, 0, None, None, None, 0, ctypes.byref(m), None) == 0
    from paper_2012_14332_gb300.binding import prior_box
    box = prior_box()
    obs = np.zeros((3, 11), dtype=np.int32)
    assert L.abc_distances(ctypes.byref(box), obs.ctypes.data_as(ctypes.c_void_p), 10, 1000, 5, 1, 0, 1, 0, None,
                           None, None) == ABC_ERR_INVALID_ARG
    # the one-call quantile form checks its arguments before any CUDA call
    eps = ctypes.c_double(0.0)
    obs_p = obs.ctypes.data_as(ctypes.c_void_p)

    def quantile(n=100, k=5, outs=(z, z, z), eps_p=ctypes.byref(eps), m_p=ctypes.byref(m), mode=1, first=0):
        return L.abc_sample_quantile(ctypes.byref(box), obs_p, 10, 1000, n, k, 1, 0, mode, first, *outs, 4, eps_p,
                                     m_p, None)
    m.value = 9
    assert quantile(k=0) == ABC_ERR_INVALID_ARG
    assert m.value == 0
    assert quantile(k=101) == ABC_ERR_INVALID_ARG
    assert quantile(n=0, k=1) == ABC_ERR_INVALID_ARG
    assert quantile(outs=(None, z, z)) == ABC_ERR_INVALID_ARG
    assert quantile(eps_p=None) == ABC_ERR_INVALID_ARG
    assert quantile(m_p=None) == ABC_ERR_INVALID_ARG
    assert quantile(mode=99) == ABC_ERR_INVALID_ARG
    assert quantile(n=2**41, k=1) == ABC_ERR_INVALID_ARG
    assert quantile(first=2**64 - 50) == ABC_ERR_INVALID_ARG
    n1, n2 = ctypes.c_uint64(7), ctypes.c_uint64(7)
    assert L.abc_sample_until(ctypes.byref(box), None, 1.0, 5, 10, 100, 1, 0, 1, 0, None, None, None, 0,
                              ctypes.byref(n1), ctypes.byref(n2), None) == ABC_ERR_INVALID_ARG
    assert "observed" in L.abc_last_error().decode()
    bad = prior_box(hi=[0.0] * 8)
    assert L.abc_sample_until(ctypes.byref(bad), None, 1.0, 5, 10, 100, 1, 0, 1, 0, None, None, None, 0,
                              ctypes.byref(n1), ctypes.byref(n2), None) == ABC_ERR_INVALID_ARG
    # flow calls on a NULL flow return before any CUDA call
    assert L.abc_maf_test_hold_products(None, 1) == ABC_ERR_INVALID_ARG
    assert "NULL" in L.abc_last_error().decode()


def test_zero_samples_is_a_no_op(L):
    # n_samples = 0 returns before any CUDA call
    from paper_2012_14332_gb300.binding import ABC_OK
    assert _call_sample(L, n=0) == ABC_OK


def test_oracle_is_not_reachable_from_the_product():
    """The CUDA package neither imports nor links the oracle."""
    pkg = os.path.join(ROOT, "paper_2012_14332_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower(), os.path.join(dirpath, f)


def test_plan_create_validates_before_any_cuda_call(L):
    from paper_2012_14332_gb300.binding import ABC_ERR_INVALID_ARG, AbcRegion, prior_box
    box = prior_box()
    obs = np.zeros((3, 11), dtype=np.int32)
    obs[0, 0] = 5
    good = dict(observed=obs.ctypes.data, T=10, N_pop=1000, eps=1.0, n_samples=10, first_index=0, stream=0,
                capacity=4, theta_in=None)

    def create(regs, n=None):
        arr = (AbcRegion * max(1, len(regs)))(*[AbcRegion(**r) for r in regs])
        h = ctypes.c_void_p()
        return L.abc_plan_create(ctypes.byref(box), arr, len(regs) if n is None else n, 1, 1, ctypes.byref(h))

    assert create([good], n=0) == ABC_ERR_INVALID_ARG
    assert create([good], n=33) == ABC_ERR_INVALID_ARG
    for bad in (dict(T=0), dict(T=5000), dict(N_pop=0), dict(eps=-1.0), dict(eps=float("nan")),
                dict(stream=2**30), dict(observed=None)):
        assert create([good, dict(good, **bad)]) == ABC_ERR_INVALID_ARG, bad
        assert "region 1" in L.abc_last_error().decode()
    big = obs.copy()
    big[:, 0] = [900, 90, 20]
    assert create([dict(good, observed=big.ctypes.data)]) == ABC_ERR_INVALID_ARG
    assert L.abc_plan_run(None, None) == ABC_ERR_INVALID_ARG
    assert L.abc_plan_destroy(None) == ABC_ERR_INVALID_ARG


def test_sequential_drivers_validate_before_any_cuda_call(L):
    """Bad configurations of the sequential drivers (one region, many regions)
    and of flow training return ABC_ERR_INVALID_ARG without touching a GPU;
    a round must keep every accepted sample (capacity >= sims_per_round)."""
    from paper_2012_14332_gb300.binding import (ABC_ERR_INVALID_ARG, AbcSmcConfig, AbcSmcRegion, AbcSmcRound,
                                                AbcSmcStreamConfig, prior_box)
    box = prior_box()
    obs = np.zeros((3, 11), dtype=np.int32)
    obs[0, 0] = 5
    op = obs.ctypes.data_as(ctypes.c_void_p)
    good = dict(rounds=3, sims_per_round=1024, eps0=10.0, eps_factor=0.7, ess_min=0.1, flow_blocks=3, flow_hidden=64,
                train_steps=10, train_batch=256, train_lr=1e-3, seed=1, capacity=1024, mode=1, defensive=0.1,
                val_fraction=0.1, train_weight_power=1.0, fresh_init=0, proposal_scale=1.0, fallback_rule=0)
    rounds = (AbcSmcRound * 16)()
    n = ctypes.c_uint64()
    s = ctypes.c_void_p(1)   # never used: validation fails first
    for bad in (dict(capacity=1023), dict(rounds=0), dict(eps_factor=1.5), dict(defensive=1.0),
                dict(val_fraction=0.6), dict(sims_per_round=0), dict(train_weight_power=0.0),
                dict(train_weight_power=1.5), dict(proposal_scale=0.4), dict(proposal_scale=4.5),
                dict(fallback_rule=2)):
        cfg = AbcSmcConfig(**dict(good, **bad))
        assert L.abc_smc_run(ctypes.byref(box), op, 10, 1000, ctypes.byref(cfg), rounds, None, None, None,
                             ctypes.byref(n), s) == ABC_ERR_INVALID_ARG, bad
    assert "capacity" in (L.abc_smc_run(ctypes.byref(box), op, 10, 1000,
                                        ctypes.byref(AbcSmcConfig(**dict(good, capacity=1))), rounds, None, None,
                                        None, ctypes.byref(n), s) and L.abc_last_error().decode())
    reg = (AbcSmcRegion * 2)(AbcSmcRegion(op, 10, 1000, 5.0, None, None, None, 0, 0, 0),
                             AbcSmcRegion(op, 10, 1000, 5.0, None, None, None, 0, 0, 0))
    for bad, shrink, nreg in ((dict(), 0, 2), (dict(), 4, 2), (dict(capacity=10), 2, 2), (dict(), 2, 0),
                              (dict(), 2, 33), (dict(proposal_scale=0.0), 2, 2)):
        cfg = AbcSmcStreamConfig(AbcSmcConfig(**dict(good, **bad)), shrink, 5)
        assert L.abc_smc_run_regions(ctypes.byref(box), reg, nreg, ctypes.byref(cfg), rounds, s) \
            == ABC_ERR_INVALID_ARG, (bad, shrink, nreg)
    # a region with capacity but no output buffers
    reg[1] = AbcSmcRegion(op, 10, 1000, 5.0, None, None, None, 8, 0, 0)
    cfg = AbcSmcStreamConfig(AbcSmcConfig(**good), 2, 5)
    assert L.abc_smc_run_regions(ctypes.byref(box), reg, 2, ctypes.byref(cfg), rounds, s) == ABC_ERR_INVALID_ARG


def test_failed_scratch_allocation_is_reported(L, monkeypatch):
    """A scratch allocation that fails (made to fail on the host) returns
    ABC_ERR_NOMEM with a message, before any kernel is launched: the calls
    that take stream-ordered scratch from the library's pool."""
    from paper_2012_14332_gb300.binding import ABC_ERR_NOMEM, prior_box
    monkeypatch.setenv("ABC_GB300_INJECT_FAULT", "alloc")
    box = prior_box()
    obs = np.zeros((3, 11), dtype=np.int32)
    obs[0, 0] = 5
    obs_p = obs.ctypes.data_as(ctypes.c_void_p)
    z = ctypes.c_void_p(16)
    eps, m = ctypes.c_double(), ctypes.c_uint64(3)
    assert L.abc_distances(ctypes.byref(box), obs_p, 10, 1000, 64, 1, 0, 1, 0, z, None, None) == ABC_ERR_NOMEM
    assert L.abc_sample_quantile(ctypes.byref(box), obs_p, 10, 1000, 64, 3, 1, 0, 1, 0, z, z, z, 4,
                                 ctypes.byref(eps), ctypes.byref(m), None) == ABC_ERR_NOMEM
    assert m.value == 0 and "injected" in L.abc_last_error().decode()
    assert L.abc_kth_smallest(z, 10, 3, ctypes.byref(eps), None) == ABC_ERR_NOMEM
    assert L.abc_select_below(z, None, 10, 1.0, 0, None, z, z, 4, ctypes.byref(m), None) == ABC_ERR_NOMEM
