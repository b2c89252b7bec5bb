"""Masked autoregressive flow (MAF) proposal for sequential ABC, float64.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import this module. The CUDA library never does.

The paper names sequential Monte Carlo ABC (Sec. 2.2, last paragraph: a
decreasing sequence of tolerances, each round's samples transformed into the
next) without fixing how the next proposal is built. The proposal here is a
density q(theta) learned from the previous round's accepted, importance
weighted samples:

  * support: the prior box, through y = logit((theta - lo) / (hi - lo)),
    with (theta - lo) / (hi - lo) held in [2^-24, 1 - 2^-24];
  * flow (Papamakarios, Pavlakou, Murray 2017): K MADE blocks (Germain, Gregor,
    Murray, Larochelle 2015), each x -> z = (x - mu(x)) exp(-alpha(x)) with
    mu_j, alpha_j depending on x_{<j} only, the order reversed between blocks;
  * base: independent standard logistic coordinates, log p(z) =
    -|z| - 2 log(1 + exp(-|z|)). The logit of a uniform variable is standard
    logistic, so the flow with zero parameters is exactly the uniform prior
    on the box, and in a coordinate where the posterior stays flat up to the
    box's edge the flow's tails can match it (a Gaussian base cannot);
  * MADE: h = relu(W1 x + b1) with mask M1[l, j] = [d_h(l) >= j + 1], outputs
    (mu, alpha_raw) = W2 h + b2 with mask M2[j, l] = [j + 1 > d_h(l)], hidden
    degrees d_h(l) = (l mod (D - 1)) + 1;
  * alpha = A tanh(alpha_raw / A), A = 6 (keeps exp(alpha) bounded);
  * log q(theta) = log p(z_K) - sum_k sum_j alpha_kj - sum_j log((hi_j - lo_j) u_j (1 - u_j));
  * importance weight of an accepted draw: w = prior(theta) / q(theta);
  * training: Adam (Kingma, Ba 2015) on the weighted mean of -log q_y(y).
"""
import numpy as np

D = 8
ALPHA_MAX = 6.0


def log_base(z):
    """Sum over coordinates of the standard logistic log density."""
    a = np.abs(np.asarray(z, dtype=np.float64))
    return (-a - 2.0 * np.log1p(np.exp(-a))).sum(axis=-1)


def base_grad(z):
    """d/dz of -log p(z) per coordinate: tanh(z / 2)."""
    return np.tanh(0.5 * np.asarray(z, dtype=np.float64))


def degrees(H, D=D):
    return (np.arange(H) % (D - 1)) + 1


def masks(H, D=D):
    """M1 [H, D] and M2 [2D, H] (rows 0..D-1 for mu, D..2D-1 for alpha)."""
    d_in = np.arange(1, D + 1)
    d_h = degrees(H, D)
    M1 = (d_h[:, None] >= d_in[None, :]).astype(np.float64)
    M2 = (d_in[:, None] > d_h[None, :]).astype(np.float64)
    return M1, np.concatenate([M2, M2], axis=0)


def init_params(rng, K=3, H=256, D=D, scale=0.1):
    """K blocks of (W1 [H, D], b1 [H], W2 [2D, H], b2 [2D]), small random weights."""
    out = []
    for _ in range(K):
        out.append(dict(W1=rng.normal(0, scale / np.sqrt(D), (H, D)), b1=np.zeros(H),
                        W2=rng.normal(0, scale / np.sqrt(H), (2 * D, H)), b2=np.zeros(2 * D)))
    return out


def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def made(x, p, M1, M2, bf16=False):
    """One MADE: returns (mu, alpha, alpha_raw, hidden pre-activation, hidden).
    bf16=True rounds the two matrix products' inputs (x, h and the weights) to
    bfloat16, the precision of a BF16 tensor-core product with FP32 sums."""
    W1, W2 = p["W1"] * M1, p["W2"] * M2
    if bf16:
        x, W1, W2 = round_bf16(x), round_bf16(W1), round_bf16(W2)
    a1 = x @ W1.T + p["b1"]
    h = np.maximum(a1, 0.0)
    out = (round_bf16(h) if bf16 else h) @ W2.T + p["b2"]
    mu = out[:, :D]
    araw = out[:, D:]
    alpha = ALPHA_MAX * np.tanh(araw / ALPHA_MAX)
    return mu, alpha, araw, a1, h


def forward(y, params, bf16=False, tau=1.0):
    """y [N, D] -> (z [N, D] after the last reversal, log q_y [N], per-block caches).
    tau > 1 evaluates the broadened proposal whose base is tau * (standard logistic)."""
    H = params[0]["W1"].shape[0]
    M1, M2 = masks(H)
    x = np.asarray(y, dtype=np.float64)
    logdet = np.zeros(x.shape[0])
    caches = []
    for p in params:
        mu, alpha, araw, a1, h = made(x, p, M1, M2, bf16)
        z = (x - mu) * np.exp(-alpha)
        logdet -= alpha.sum(axis=1)
        caches.append(dict(x=x, mu=mu, alpha=alpha, araw=araw, a1=a1, h=h, z=z))
        x = z[:, ::-1]
    logq = log_base(x / tau) - D * np.log(tau) + logdet
    return x, logq, caches


def inverse(u, params, bf16=False, tau=1.0):
    """Base draws u [N, D] (standard logistic) -> (y [N, D], log q_y [N]) by the
    sequential inverse of the flow whose base is tau * (standard logistic)."""
    H = params[0]["W1"].shape[0]
    M1, M2 = masks(H)
    x = tau * np.asarray(u, dtype=np.float64)
    logq = log_base(x / tau) - D * np.log(tau)
    for p in reversed(params):
        z = x[:, ::-1]
        xin = np.zeros_like(z)
        for j in range(D):
            mu, alpha, _, _, _ = made(xin, p, M1, M2, bf16)
            xin[:, j] = z[:, j] * np.exp(alpha[:, j]) + mu[:, j]
        mu, alpha, _, _, _ = made(xin, p, M1, M2, bf16)
        logq -= alpha.sum(axis=1)
        x = xin
    return x, logq


def to_theta(y, lo, hi):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) / (1.0 + np.exp(-y))


def to_y(theta, lo, hi):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = (np.asarray(theta, dtype=np.float64) - lo) / (hi - lo)
    # a point on the box's edge is read as 2^-24 of the width inside
    u = np.clip(u, 2.0**-24, 1 - 2.0**-24)
    return np.log(u) - np.log1p(-u)


def log_jacobian_y(y, lo, hi):
    """sum_j log |d theta_j / d y_j| = sum_j log((hi - lo) s (1 - s)), s = sigmoid(y)."""
    w = np.asarray(hi, dtype=np.float64) - np.asarray(lo, dtype=np.float64)
    return (np.log(w) - np.logaddexp(0, -y) - np.logaddexp(0, y)).sum(axis=1)


def log_q_theta(theta, params, lo, hi, bf16=False, tau=1.0):
    y = to_y(theta, lo, hi)
    _, logq_y, _ = forward(y, params, bf16, tau)
    return logq_y - log_jacobian_y(y, lo, hi)


def loss_and_grad(y, w, params, bf16=False, with_scale=False):
    """Weighted mean of -log q_y(y) and its gradient with respect to every parameter.

    bf16=True follows the precision of a BF16 tensor-core backward pass with
    FP32 sums: the forward pass as made(bf16=True); every operand entering a
    backward matrix product is rounded to bfloat16 (g_out = (g_mu, g_alpha_raw)
    and the masked W2 for g_h = g_out W2; g_a1 and the masked W1 for
    g_x = g_a1 W1; h, g_out, g_a1 and x for the weight gradients; g_a1 for
    db1 = sum of g_a1 over rows), db2 stays the sum of the unrounded g_out.
    The per-row weights enter unnormalised (w, not w / sum w), as they do on
    a device that sums w (-log q) over the rows, and the gradient is divided
    by sum w at the end: rounding to bfloat16 commutes with a power-of-two
    scale only, so the scale must be applied where the device applies it.

    with_scale=True also returns, per gradient entry, the sum over rows of the
    absolute values of its terms (each product's |a| |b|, divided by sum w):
    the natural scale of that entry's rounding error."""
    H = params[0]["W1"].shape[0]
    M1, M2 = masks(H)
    w = np.asarray(w, dtype=np.float64)
    W = w.sum()
    rb = round_bf16 if bf16 else (lambda a: a)
    wr = w if bf16 else w / W                      # row weights in the backward pass
    zK, logq, caches = forward(y, params, bf16=bf16)
    loss = -(w * logq).sum() / W
    g_x = wr[:, None] * base_grad(zK)              # d loss / d (final x)
    grads = [None] * len(params)
    scales = [None] * len(params)
    for k in reversed(range(len(params))):
        c, p = caches[k], params[k]
        g_z = g_x[:, ::-1]                         # undo the reversal after block k
        e = np.exp(-c["alpha"])
        g_xdirect = g_z * e
        g_mu = -g_z * e
        # d loss / d alpha: -g_z z (through z = (x - mu) e^-alpha) + w (log-det term)
        g_alpha = -g_z * c["z"] + wr[:, None]
        g_araw = g_alpha * (1.0 - (c["alpha"] / ALPHA_MAX) ** 2)
        g_out = np.concatenate([g_mu, g_araw], axis=1)          # [N, 2D]
        gob, hb, xb = rb(g_out), rb(c["h"]), rb(c["x"])
        W2m, W1m = rb(p["W2"] * M2), rb(p["W1"] * M1)
        gW2 = (gob.T @ hb) * M2
        gb2 = g_out.sum(axis=0)
        g_h = gob @ W2m
        g_a1 = rb(g_h * (c["a1"] > 0))
        gW1 = (g_a1.T @ xb) * M1
        gb1 = g_a1.sum(axis=0)
        g_x = g_xdirect + g_a1 @ W1m
        grads[k] = dict(W1=gW1, b1=gb1, W2=gW2, b2=gb2)
        if with_scale:
            scales[k] = dict(W1=(np.abs(g_a1).T @ np.abs(xb)) * M1, b1=np.abs(g_a1).sum(axis=0),
                             W2=(np.abs(gob).T @ np.abs(hb)) * M2, b2=np.abs(g_out).sum(axis=0))
    if bf16:
        grads = [{key: v / W for key, v in g.items()} for g in grads]
    if with_scale:
        sw = W if bf16 else 1.0
        scales = [{key: v / sw for key, v in g.items()} for g in scales]
        return loss, grads, scales
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma, Ba 2015) in place; state: dict(t, m, v)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    if "m" not in state:
        state["m"] = [{k: np.zeros_like(v) for k, v in p.items()} for p in params]
        state["v"] = [{k: np.zeros_like(v) for k, v in p.items()} for p in params]
    for p, g, m, v in zip(params, grads, state["m"], state["v"]):
        for key in p:
            m[key] = b1 * m[key] + (1 - b1) * g[key]
            v[key] = b2 * v[key] + (1 - b2) * g[key] ** 2
            mhat = m[key] / (1 - b1 ** t)
            vhat = v[key] / (1 - b2 ** t)
            p[key] = p[key] - lr * mhat / (np.sqrt(vhat) + eps)


def ess_fraction(w):
    w = np.asarray(w, dtype=np.float64)
    return (w.sum() ** 2) / (w ** 2).sum() / len(w)


def flat(params):
    """Parameters in the library's order: per block W1, b1, W2, b2 (row-major)."""
    return np.concatenate([np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"]]) for p in params])


def unflat(v, K, H):
    out, o = [], 0
    for _ in range(K):
        W1 = v[o:o + H * D].reshape(H, D); o += H * D
        b1 = v[o:o + H]; o += H
        W2 = v[o:o + 2 * D * H].reshape(2 * D, H); o += 2 * D * H
        b2 = v[o:o + 2 * D]; o += 2 * D
        out.append(dict(W1=W1.astype(np.float64), b1=b1.astype(np.float64), W2=W2.astype(np.float64),
                        b2=b2.astype(np.float64)))
    return out
