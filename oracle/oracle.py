"""ctypes wrapper of the C oracle (test infrastructure only).

Every function here marshals numpy arrays into ``abc_oracle.c`` and back; the
arithmetic lives in the C file, which cites the paper passage for each step.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Plain IEEE binary32 arithmetic: no contraction into FMA (aarch64 GCC
# contracts by default), no fast-math, no vector intrinsics.
CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
          "-pthread", "-Wall", "-Wextra"]

PAPER_LO = np.zeros(8, dtype=np.float32)
PAPER_HI = np.array([1, 100, 2, 1, 1, 1, 1, 2], dtype=np.float32)  # Sec. 2.1, Eq. 2


def build(force=False):
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, plain C11)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "abc_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc"] + CFLAGS + ["-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            u32p, f32p, i32p = P(ctypes.c_uint32), P(ctypes.c_float), P(ctypes.c_int32)
            u64p, f64p = P(ctypes.c_uint64), P(ctypes.c_double)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oracle_uniform.argtypes = [ctypes.c_uint32]
            L.oracle_uniform.restype = ctypes.c_float
            L.oracle_log2x.argtypes = [ctypes.c_float]
            L.oracle_log2x.restype = ctypes.c_float
            L.oracle_exp2x.argtypes = [ctypes.c_float]
            L.oracle_exp2x.restype = ctypes.c_float
            L.oracle_sincospix.argtypes = [ctypes.c_float, f32p, f32p]
            L.oracle_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, f32p]
            L.oracle_day_pair_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                                  ctypes.c_uint32, f32p]
            L.oracle_prior_draw.argtypes = [f32p, f32p, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint64, f32p]
            L.oracle_clamp_count.argtypes = [ctypes.c_float, ctypes.c_int32]
            L.oracle_clamp_count.restype = ctypes.c_int32
            L.oracle_infection_rate.argtypes = [f32p, ctypes.c_int32]
            L.oracle_infection_rate.restype = ctypes.c_float
            L.oracle_hazard.argtypes = [i32p, f32p, ctypes.c_int64, f32p]
            L.oracle_step.argtypes = [i32p, f32p, ctypes.c_int64, f32p, ctypes.c_int, i32p, i32p]
            L.oracle_init_state.argtypes = [f32p, i32p, ctypes.c_int64, i32p]
            L.oracle_init_state.restype = ctypes.c_int
            L.oracle_simulate.argtypes = [f32p, i32p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                          ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, i32p]
            L.oracle_simulate.restype = ctypes.c_int
            L.oracle_sq_distance.argtypes = [i32p, i32p, ctypes.c_int32]
            L.oracle_sq_distance.restype = ctypes.c_uint64
            L.oracle_distance_from_sq.argtypes = [ctypes.c_uint64]
            L.oracle_distance_from_sq.restype = ctypes.c_double
            L.oracle_abc.argtypes = [f32p, f32p, i32p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_int, ctypes.c_int, u64p, f32p, f64p, ctypes.c_uint64,
                                     u64p, f64p]
            L.oracle_abc.restype = ctypes.c_int
            for nm in ("oracle_log2x_batch", "oracle_exp2x_batch"):
                getattr(L, nm).argtypes = [f32p, f32p, ctypes.c_uint64]
            L.oracle_sincospix_batch.argtypes = [f32p, f32p, f32p, ctypes.c_uint64]
            L.oracle_uniform_batch.argtypes = [u32p, f32p, ctypes.c_uint64]
            L.oracle_normals_batch.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                               ctypes.c_uint64, ctypes.c_uint32, f32p]
            L.oracle_prior_batch.argtypes = [f32p, f32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                             ctypes.c_uint64, f32p]
            L.oracle_step_batch.argtypes = [i32p, f32p, ctypes.c_int64, f32p, ctypes.c_int, ctypes.c_uint64,
                                            i32p, i32p]
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(ctr, ctypes.c_uint32), _ptr(key, ctypes.c_uint32),
                               _ptr(out, ctypes.c_uint32))
    return out


def uniform(w):
    return np.float32(lib().oracle_uniform(int(w)))


def log2x(x):
    return np.float32(lib().oracle_log2x(float(x)))


def exp2x(y):
    return np.float32(lib().oracle_exp2x(float(y)))


def sincospix(v):
    s, c = ctypes.c_float(), ctypes.c_float()
    lib().oracle_sincospix(float(v), ctypes.byref(s), ctypes.byref(c))
    return np.float32(s.value), np.float32(c.value)


def box_muller(w_radius, w_angle):
    z = np.zeros(2, dtype=np.float32)
    lib().oracle_box_muller(int(w_radius), int(w_angle), _ptr(z, ctypes.c_float))
    return z


def day_pair_normals(seed, stream, i, k):
    z = np.zeros(10, dtype=np.float32)
    lib().oracle_day_pair_normals(seed, stream, i, k, _ptr(z, ctypes.c_float))
    return z


def prior_draw(seed, stream, i, lo=PAPER_LO, hi=PAPER_HI):
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    th = np.zeros(8, dtype=np.float32)
    lib().oracle_prior_draw(_ptr(lo, ctypes.c_float), _ptr(hi, ctypes.c_float), seed, stream, i,
                            _ptr(th, ctypes.c_float))
    return th


def clamp_count(x, c):
    return int(lib().oracle_clamp_count(float(np.float32(x)), int(c)))


def infection_rate(theta, U):
    th = np.ascontiguousarray(theta, dtype=np.float32)
    return np.float32(lib().oracle_infection_rate(_ptr(th, ctypes.c_float), int(U)))


def hazard(X, theta, P):
    X = np.ascontiguousarray(X, dtype=np.int32)
    th = np.ascontiguousarray(theta, dtype=np.float32)
    h = np.zeros(5, dtype=np.float32)
    lib().oracle_hazard(_ptr(X, ctypes.c_int32), _ptr(th, ctypes.c_float), int(P), _ptr(h, ctypes.c_float))
    return h


def step(X, theta, P, z, variance_literal=False):
    """One day from state X with the five normals z (h order) -> (n[5], Y[6])."""
    X = np.ascontiguousarray(X, dtype=np.int32)
    th = np.ascontiguousarray(theta, dtype=np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    n = np.zeros(5, dtype=np.int32)
    Y = np.zeros(6, dtype=np.int32)
    lib().oracle_step(_ptr(X, ctypes.c_int32), _ptr(th, ctypes.c_float), int(P), _ptr(z, ctypes.c_float),
                      int(bool(variance_literal)), _ptr(n, ctypes.c_int32), _ptr(Y, ctypes.c_int32))
    return n, Y


def init_state(theta, ard0, P):
    th = np.ascontiguousarray(theta, dtype=np.float32)
    a = np.ascontiguousarray(ard0, dtype=np.int32)
    X = np.zeros(6, dtype=np.int32)
    rc = lib().oracle_init_state(_ptr(th, ctypes.c_float), _ptr(a, ctypes.c_int32), int(P),
                                 _ptr(X, ctypes.c_int32))
    if rc != 0:
        raise ValueError("A0 + R0 + D0 exceeds the population")
    return X


def simulate(theta, ard0, T, P, seed, stream, i, variance_literal=False):
    """Trajectory [T+1, 6] (S, I, A, R, D, Ru) of sample index i with the given theta."""
    th = np.ascontiguousarray(theta, dtype=np.float32)
    a = np.ascontiguousarray(ard0, dtype=np.int32)
    traj = np.zeros((T + 1, 6), dtype=np.int32)
    rc = lib().oracle_simulate(_ptr(th, ctypes.c_float), _ptr(a, ctypes.c_int32), int(T), int(P),
                               seed, stream, i, int(bool(variance_literal)), _ptr(traj, ctypes.c_int32))
    if rc != 0:
        raise ValueError("invalid initial condition")
    return traj


def sq_distance(traj, observed):
    traj = np.ascontiguousarray(traj, dtype=np.int32)
    observed = np.ascontiguousarray(observed, dtype=np.int32)
    T = observed.shape[1] - 1
    return int(lib().oracle_sq_distance(_ptr(traj, ctypes.c_int32), _ptr(observed, ctypes.c_int32), T))


def distance_from_sq(acc):
    return float(lib().oracle_distance_from_sq(int(acc)))


def abc(observed, P, eps, n_samples, seed, stream=0, first_index=0, lo=PAPER_LO, hi=PAPER_HI,
        capacity=None, n_threads=0, variance_literal=False, want_all=False):
    """ABC rejection over sample indices [first_index, first_index + n_samples).

    Returns dict(idx, theta, dist, n_accepted[, dist_all]) with the accepted
    samples sorted by index.
    """
    observed = np.ascontiguousarray(observed, dtype=np.int32)
    T = observed.shape[1] - 1
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    if capacity is None:
        capacity = max(1, n_samples)
    idx = np.zeros(capacity, dtype=np.uint64)
    th = np.zeros((capacity, 8), dtype=np.float32)
    dist = np.zeros(capacity, dtype=np.float64)
    nacc = ctypes.c_uint64(0)
    dist_all = np.zeros(n_samples if want_all else 0, dtype=np.float64)
    rc = lib().oracle_abc(_ptr(lo, ctypes.c_float), _ptr(hi, ctypes.c_float), _ptr(observed, ctypes.c_int32),
                          int(T), int(P), float(eps), int(n_samples), seed, stream, first_index,
                          int(bool(variance_literal)), int(n_threads),
                          _ptr(idx, ctypes.c_uint64), _ptr(th, ctypes.c_float), _ptr(dist, ctypes.c_double),
                          int(capacity), ctypes.byref(nacc),
                          _ptr(dist_all, ctypes.c_double) if want_all else None)
    if rc < 0:
        raise RuntimeError("oracle_abc failed with status %d" % rc)
    n = int(nacc.value)
    m = min(n, capacity)
    out = dict(idx=idx[:m], theta=th[:m], dist=dist[:m], n_accepted=n, overflow=(rc == 1))
    if want_all:
        out["dist_all"] = dist_all
    return out


def log2x_batch(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().oracle_log2x_batch(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), x.size)
    return y


def exp2x_batch(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().oracle_exp2x_batch(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), x.size)
    return y


def sincospix_batch(v):
    v = np.ascontiguousarray(v, dtype=np.float32)
    s = np.empty_like(v)
    c = np.empty_like(v)
    lib().oracle_sincospix_batch(_ptr(v, ctypes.c_float), _ptr(s, ctypes.c_float), _ptr(c, ctypes.c_float),
                                 v.size)
    return s, c


def uniform_batch(w):
    w = np.ascontiguousarray(w, dtype=np.uint32)
    u = np.empty(w.shape, dtype=np.float32)
    lib().oracle_uniform_batch(_ptr(w, ctypes.c_uint32), _ptr(u, ctypes.c_float), w.size)
    return u


def normals_batch(seed, stream, first, n, k):
    """[n, 10] normals of day-pair k for samples first .. first+n-1."""
    z = np.empty((n, 10), dtype=np.float32)
    lib().oracle_normals_batch(seed, stream, first, n, k, _ptr(z, ctypes.c_float))
    return z


def prior_batch(seed, stream, first, n, lo=PAPER_LO, hi=PAPER_HI):
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    th = np.empty((n, 8), dtype=np.float32)
    lib().oracle_prior_batch(_ptr(lo, ctypes.c_float), _ptr(hi, ctypes.c_float), seed, stream, first, n,
                             _ptr(th, ctypes.c_float))
    return th


def step_batch(X, theta, P, z, variance_literal=False):
    """One step for each row: X [m,6], theta [m,8], z [m,5] -> (n [m,5], Y [m,6])."""
    X = np.ascontiguousarray(X, dtype=np.int32)
    th = np.ascontiguousarray(theta, dtype=np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    m = X.shape[0]
    assert th.shape == (m, 8) and z.shape == (m, 5) and X.shape == (m, 6)
    n = np.empty((m, 5), dtype=np.int32)
    Y = np.empty((m, 6), dtype=np.int32)
    lib().oracle_step_batch(_ptr(X, ctypes.c_int32), _ptr(th, ctypes.c_float), int(P), _ptr(z, ctypes.c_float),
                            int(bool(variance_literal)), m, _ptr(n, ctypes.c_int32), _ptr(Y, ctypes.c_int32))
    return n, Y


__all__ = ["build", "lib", "philox4x32_10", "uniform", "log2x", "exp2x", "sincospix", "box_muller",
           "day_pair_normals", "prior_draw", "clamp_count", "infection_rate", "hazard", "step",
           "init_state", "simulate", "sq_distance", "distance_from_sq", "abc", "PAPER_LO", "PAPER_HI",
           "log2x_batch", "exp2x_batch", "sincospix_batch", "uniform_batch", "normals_batch", "prior_batch",
           "step_batch"]
