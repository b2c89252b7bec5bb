"""Two-sample tests between an importance-weighted sample and a plain one,
used by the GPU tests of the sequential samplers (plain numpy/scipy)."""
import numpy as np
from scipy import stats


def sandwich_ks(x, w, y):
    """sup |F_w - G| between a self-normalised importance-weighted sample and a
    plain one, with a p-value from the Kolmogorov distribution at the smallest
    local effective size n_eff(t) = F(1 - F) / Var F_w(t), Var from the
    sandwich (delta-method) form sum w_i^2 (1{x_i <= t} - F_w(t))^2 / (sum w)^2.
    Where the large weights gather in one tail, (sum w)^2 / sum w^2 overstates
    the precision of F_w there; the local size does not."""
    o = np.argsort(x)
    xs, ws = x[o], w[o] / w.sum()
    ys = np.sort(y)
    grid = np.concatenate([xs, ys])
    cw = np.concatenate([[0.0], np.cumsum(ws)])
    k = np.searchsorted(xs, grid, side="right")
    Fw = cw[k]
    G = np.searchsorted(ys, grid, side="right") / len(ys)
    D = np.max(np.abs(Fw - G))
    # sandwich variance at the grid points: sum_i w_i^2 (1{x_i <= t} - F)^2
    c2 = np.concatenate([[0.0], np.cumsum(ws ** 2)])
    var = (1 - Fw) ** 2 * c2[k] + Fw ** 2 * (c2[-1] - c2[k])
    mid = (Fw > 0.05) & (Fw < 0.95)
    ne = np.min(Fw[mid] * (1 - Fw[mid]) / np.maximum(var[mid], 1e-300)) if mid.any() else 1.0 / c2[-1]
    en = np.sqrt(ne * len(y) / (ne + len(y)))
    return D, stats.kstwobign.sf(D * en), ne


def weighted_ks(x, w, y):
    """sup |F_w - G| between a weighted sample (n_eff = ESS) and a plain one,
    with the asymptotic Kolmogorov p-value."""
    o = np.argsort(x)
    xs, ws = x[o], w[o] / w.sum()
    ys = np.sort(y)
    grid = np.concatenate([xs, ys])
    Fw = np.concatenate([[0.0], np.cumsum(ws)])[np.searchsorted(xs, grid, side="right")]
    G = np.searchsorted(ys, grid, side="right") / len(ys)
    D = np.max(np.abs(Fw - G))
    ne = w.sum() ** 2 / (w ** 2).sum()
    en = np.sqrt(ne * len(y) / (ne + len(y)))
    return D, stats.kstwobign.sf(D * en)


def cdf_z_scores(x, w, y, probs=(0.1, 0.25, 0.5, 0.75, 0.9)):
    """z-scores of the weighted CDF F_w against a plain sample y at y's
    quantiles t_p: (F_w(t) - G(t)) / sqrt(Var F_w(t) + G (1 - G) / m), Var from
    the sandwich form (self-normalised importance sampling) and the plain
    ECDF's binomial variance. Each is asymptotically N(0, 1) when both samples
    follow one distribution, whatever the weights."""
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    ys = np.sort(y)
    out = []
    for p in probs:
        t = ys[min(len(ys) - 1, int(p * len(ys)))]
        below = x <= t
        Fw = wn[below].sum()
        G = np.searchsorted(ys, t, side="right") / len(ys)
        var = (wn ** 2 * (below - Fw) ** 2).sum() + G * (1 - G) / len(ys)
        out.append((Fw - G) / np.sqrt(var))
    return np.array(out)


def weighted_mean_z(x, w, y):
    """(weighted mean - plain mean) / sqrt(sandwich variance + plain variance / m)."""
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    mw = (wn * x).sum()
    return (mw - y.mean()) / np.sqrt((wn ** 2 * (x - mw) ** 2).sum() + y.var() / len(y))


def posterior_error(x, w, y, probs=(0.1, 0.25, 0.5, 0.75, 0.9)):
    """Accuracy of an importance-weighted sample x (weights w) against a plain
    sample y of the target, one coordinate: (|mean difference| in units of the
    plain standard deviation, its standard error in the same units, max
    |F_w(t_p) - G(t_p)| over y's quantiles t_p, the standard error there),
    standard errors from the sandwich variance and the plain sample's."""
    wn = np.asarray(w, dtype=np.float64) / np.sum(w)
    sd = y.std()
    mw = (wn * x).sum()
    dm = abs(mw - y.mean()) / sd
    se_m = np.sqrt((wn ** 2 * (x - mw) ** 2).sum() + y.var() / len(y)) / sd
    ys = np.sort(y)
    dc, se_c = 0.0, 0.0
    for p in probs:
        t = ys[min(len(ys) - 1, int(p * len(ys)))]
        below = x <= t
        Fw = wn[below].sum()
        G = np.searchsorted(ys, t, side="right") / len(ys)
        se = np.sqrt((wn ** 2 * (below - Fw) ** 2).sum() + G * (1 - G) / len(ys))
        if abs(Fw - G) - 4 * se > dc - 4 * se_c:
            dc, se_c = abs(Fw - G), se
    return dm, se_m, dc, se_c


def assert_posterior_close(x, w, y, tol_mean=0.05, tol_cdf=0.02, k=4.0, tag=""):
    """Every coordinate: |mean difference| <= tol_mean plain sd + k SE and
    max CDF difference at five quantiles <= tol_cdf + k SE."""
    for j in range(x.shape[1]):
        dm, se_m, dc, se_c = posterior_error(x[:, j], w, y[:, j])
        assert dm <= tol_mean + k * se_m, (tag, j, dm, se_m)
        assert dc <= tol_cdf + k * se_c, (tag, j, dc, se_c)
