"""Population Monte Carlo ABC (plain SMC-ABC), float64.

TEST INFRASTRUCTURE: only tests/ may import this module; the CUDA library
never does.

The paper names SMC-ABC (Sec. 2.2, last paragraph) without its steps; this is
the population Monte Carlo scheme of Beaumont, Cornuet, Marin and Robert
(2009), the perturbation-kernel form of Toni et al. (2009) with the kernel
variance they derive:

  round 0: rejection from the prior at eps_0, weights 1;
  round t: eps_t = factor * eps_{t-1}; proposals theta = theta_j + L z with
           parent j drawn with probability w_j / sum w, z ~ N(0, I) and
           L L^T = Sigma = 2 Cov_w(previous particles); a proposal outside the
           prior box has prior density 0 and is not simulated; an accepted
           particle gets w = prior(theta) / sum_j w_j N(theta; theta_j, Sigma)
           (the constant prior and the Gaussian normaliser cancel on
           normalisation: w proportional to 1 / sum_j w_j exp(-|L^-1 (theta - theta_j)|^2 / 2)).
"""
import numpy as np


def weighted_cov(theta, w):
    w = np.asarray(w, dtype=np.float64) / np.sum(w)
    m = w @ theta
    d = theta - m
    return (d * w[:, None]).T @ d


def kernel_factor(theta, w, jitter=1e-12):
    """L with L L^T = 2 Cov_w (jitter on the diagonal if not positive definite)."""
    S = 2.0 * weighted_cov(np.asarray(theta, dtype=np.float64), w)
    scale = np.mean(np.diag(S)) if np.mean(np.diag(S)) > 0 else 1.0
    for k in range(8):
        try:
            return np.linalg.cholesky(S + np.eye(len(S)) * jitter * scale * 10 ** k)
        except np.linalg.LinAlgError:
            continue
    raise np.linalg.LinAlgError("covariance not positive definite")


def parent_uniform(w0, w1):
    """The parent draw's uniform in [0, 1) from two 32-bit random words: the
    top 27 bits of w0 and the top 26 bits of w1 form a 53-bit integer, scaled
    by 2^-53 (a double with every value k 2^-53, k < 2^53, equally likely)."""
    w0 = np.asarray(w0, dtype=np.uint64)
    w1 = np.asarray(w1, dtype=np.uint64)
    k = ((w0 >> np.uint64(5)) << np.uint64(26)) | (w1 >> np.uint64(6))
    return k.astype(np.float64) * 2.0 ** -53


def propose(theta, w, L, u, z, lo, hi):
    """Parents from uniforms u (inverse CDF of the cumulative weights), moves
    L z; rows outside the box become NaN."""
    cw = np.cumsum(np.asarray(w, dtype=np.float64))
    j = np.minimum(np.searchsorted(cw, u * cw[-1], side="right"), len(cw) - 1)
    out = theta[j] + z @ L.T
    bad = np.any((out < lo) | (out > hi), axis=1)
    out[bad] = np.nan
    return out, j


def weights(new, old, w_old, L):
    """Unnormalised w_i = 1 / sum_j w_j exp(-|L^-1 (new_i - old_j)|^2 / 2)."""
    Li = np.linalg.inv(L)
    a = np.asarray(new, dtype=np.float64) @ Li.T
    b = np.asarray(old, dtype=np.float64) @ Li.T
    d2 = (a ** 2).sum(1)[:, None] + (b ** 2).sum(1)[None, :] - 2 * a @ b.T
    return 1.0 / (np.exp(-0.5 * np.maximum(d2, 0.0)) @ np.asarray(w_old, dtype=np.float64))
