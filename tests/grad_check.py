"""Element-wise comparison of a flow gradient with the oracle's bf16-mode gradient.

The oracle's bf16 mode (maf_oracle.loss_and_grad(bf16=True)) rounds to
bfloat16 exactly the operands that enter a BF16 tensor-core product on the
device and keeps everything else in float64. What is left between the device
and that reference is FP32 against FP64 arithmetic: FP32 sums, FP32
elementwise math and the occasional operand that lands on the other side of a
bfloat16 rounding boundary (at most a 2^-7 relative change of one term). Each of
these is a small multiple of one term's magnitude, so every entry is bounded
relative to its own error scale, the sum over rows of the absolute values of
its terms (with_scale=True), not relative to its value: an entry whose terms
cancel can be much smaller than its rounding error.

Bounds (err = |g - g_ref| / scale over entries with scale > 0):
  max    <= 2^-7
  p99    <= 2e-4
  median <= 2e-6
and g == 0 exactly where scale == 0 (masked weights, hidden units that are
never active). The max bound is one bfloat16 ulp (2^-7 of the value) of a
single term as large as the whole scale: one operand rounded the other way
moves its term by at most that much. Measured on a GB300 at the tested
shapes: max 1.5e-3 (a row that dominates its entry and whose block input sat
on a rounding boundary), p99 <= 2.8e-5, median <= 2e-7; a float32 emulation
of the device's arithmetic stays within 5e-5. A sign or a factor of two on
one block's db1, one 16-column group of dW2 or one input column of dW1 dropped
gives max errors of 0.1 to 2 (pinned on the CPU in test_oracle_maf.py).
"""
import numpy as np

MAX = 2.0 ** -7
P99 = 2e-4
MEDIAN = 2e-6


def gradient_errors(g, g_ref, scale):
    """(err over entries with scale > 0, entries with scale == 0 that are not 0)."""
    g = np.asarray(g, dtype=np.float64)
    nz = scale > 0
    err = np.abs(g[nz] - g_ref[nz]) / scale[nz]
    return err, int(np.count_nonzero(g[~nz]))


def summary(err):
    return float(np.median(err)), float(np.quantile(err, 0.99)), float(err.max())


def gradient_close(g, g_ref, scale):
    """True when g meets every bound against (g_ref, scale)."""
    err, stray = gradient_errors(g, g_ref, scale)
    med, p99, mx = summary(err)
    return stray == 0 and med <= MEDIAN and p99 <= P99 and mx <= MAX
