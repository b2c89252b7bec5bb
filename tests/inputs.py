"""Seeded synthetic inputs shared by the oracle-side and CUDA-side tests.

Holds no arithmetic of the method: only random states, parameter vectors and
index ranges drawn with numpy's own generator, plus loaders for the stored
workloads under ``tests/golden`` (which the oracle wrote).
"""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

PAPER_LO = np.zeros(8, dtype=np.float32)
PAPER_HI = np.array([1, 100, 2, 1, 1, 1, 1, 2], dtype=np.float32)


def rng(seed):
    return np.random.default_rng(seed)


def random_thetas(seed, m, lo=PAPER_LO, hi=PAPER_HI):
    g = rng(seed)
    return (lo + (hi - lo) * g.random((m, 8))).astype(np.float32)


def random_states(seed, m, P):
    """m states [S, I, A, R, D, Ru] with sum P (random composition)."""
    g = rng(seed)
    X = np.zeros((m, 6), dtype=np.int64)
    for j in range(m):
        cuts = np.sort(g.integers(0, P + 1, size=5))
        parts = np.diff(np.concatenate([[0], cuts, [P]]))
        X[j] = parts
    return X.astype(np.int32)


def load_workloads():
    with open(os.path.join(GOLDEN, "workloads.json")) as f:
        return json.load(f)


def workload(name):
    w = load_workloads()[name]
    w = dict(w)
    w["observed"] = np.array(w["observed"], dtype=np.int32)
    return w
