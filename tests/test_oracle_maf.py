"""Pins of the float64 MAF proposal oracle against what the mathematics of a
normalising flow fixes: exact invertibility, the log-determinant against a
numerical Jacobian, triangular (autoregressive) Jacobians, normalisation by
importance sampling, gradients against finite differences, Adam's closed-form
first step, the zero flow equal to the uniform prior, and maximum likelihood
recovering a known density."""
import numpy as np
import pytest

from oracle import maf_oracle as maf

H_SMALL = 32


@pytest.fixture
def params():
    return maf.init_params(np.random.default_rng(0), K=3, H=H_SMALL, scale=0.8)


def test_masks_are_autoregressive():
    M1, M2 = maf.masks(256)
    # output j may depend on input i only through a path i -> l -> j with i < j
    dep = (M2[:8] @ M1) > 0
    assert not np.any(np.triu(dep))          # no dependence on inputs >= j
    assert np.all(dep[np.tril_indices(8, -1)])  # every earlier input reaches j


def test_base_is_the_standard_logistic():
    """The base density integrates to 1, has variance pi^2 / 3 per coordinate
    and is the law of logit(U) for uniform U; its score is tanh(z / 2)."""
    z = np.linspace(-40, 40, 400001)
    p = np.exp(maf.log_base(z[:, None]))
    assert abs(np.trapezoid(p, z) - 1) < 1e-9
    assert abs(np.trapezoid(p * z ** 2, z) - np.pi ** 2 / 3) < 1e-6
    u = np.random.default_rng(11).uniform(size=200000)
    from scipy import stats
    assert stats.kstest(np.log(u) - np.log1p(-u), "logistic").pvalue > 1e-3
    zz = np.array([-3.0, -0.5, 0.0, 0.7, 5.0])
    num = -(maf.log_base((zz + 1e-6)[:, None]) - maf.log_base((zz - 1e-6)[:, None])) / 2e-6
    assert np.allclose(maf.base_grad(zz), num, atol=1e-8)


def test_zero_flow_is_the_uniform_prior():
    lo = np.zeros(8)
    hi = np.array([1, 100, 2, 1, 1, 1, 1, 2.0])
    params = maf.init_params(np.random.default_rng(0), K=3, H=H_SMALL, scale=0.0)
    th = lo + (hi - lo) * np.random.default_rng(12).uniform(0.01, 0.99, size=(50, 8))
    assert np.allclose(maf.log_q_theta(th, params, lo, hi), -np.log(np.prod(hi - lo)), atol=1e-9)


def test_inverse_roundtrip(params):
    u = np.random.default_rng(1).logistic(size=(200, 8))
    y, logq_inv = maf.inverse(u, params)
    z, logq_fwd, _ = maf.forward(y, params)
    assert np.allclose(z, u, atol=1e-10)
    assert np.allclose(logq_inv, logq_fwd, atol=1e-10)


def _full_map(y, params):
    z, _, _ = maf.forward(y[None, :], params)
    return z[0]


def test_logdet_matches_numerical_jacobian(params):
    rng = np.random.default_rng(2)
    for _ in range(5):
        y = rng.normal(size=8)
        J = np.zeros((8, 8))
        h = 1e-6
        for i in range(8):
            e = np.zeros(8)
            e[i] = h
            J[:, i] = (_full_map(y + e, params) - _full_map(y - e, params)) / (2 * h)
        z, logq, _ = maf.forward(y[None, :], params)
        logdet = logq[0] - maf.log_base(z[0])
        assert np.isclose(np.linalg.slogdet(J)[1], logdet, atol=1e-6)


def test_each_block_is_triangular(params):
    M1, M2 = maf.masks(H_SMALL)
    x = np.random.default_rng(3).normal(size=8)
    for p in params:
        J = np.zeros((8, 8))
        for i in range(8):
            e = np.zeros(8)
            e[i] = 1e-6
            mu1, a1, *_ = maf.made((x + e)[None], p, M1, M2)
            mu0, a0, *_ = maf.made((x - e)[None], p, M1, M2)
            z1 = ((x + e) - mu1[0]) * np.exp(-a1[0])
            z0 = ((x - e) - mu0[0]) * np.exp(-a0[0])
            J[:, i] = (z1 - z0) / 2e-6
        assert np.allclose(np.triu(J, 1), 0, atol=1e-9)


def test_density_is_normalised():
    """The integral of q is 1: E_{y~p}[q(y)/p(y)] with p the logistic of scale
    2 per coordinate, wider than q, so the importance ratios stay bounded."""
    params = maf.init_params(np.random.default_rng(9), K=3, H=H_SMALL, scale=0.3)
    y = np.random.default_rng(4).logistic(size=(400_000, 8)) * 2.0
    _, logq, _ = maf.forward(y, params)
    logp = maf.log_base(y / 2.0) - 8 * np.log(2)
    r = np.exp(logq - logp)
    assert abs(r.mean() - 1) < 5 * r.std() / np.sqrt(len(r))
    assert r.std() / np.sqrt(len(r)) < 0.02


def test_theta_density_change_of_variables(params):
    lo = np.zeros(8)
    hi = np.array([1, 100, 2, 1, 1, 1, 1, 2.0])
    rng = np.random.default_rng(5)
    th = lo + (hi - lo) * rng.uniform(0.05, 0.95, size=(20, 8))
    y = maf.to_y(th, lo, hi)
    assert np.allclose(maf.to_theta(y, lo, hi), th)
    # d theta_j / d y_j numerically
    h = 1e-6
    num = np.log(np.abs((maf.to_theta(y + h, lo, hi) - maf.to_theta(y - h, lo, hi)) / (2 * h))).sum(axis=1)
    assert np.allclose(maf.log_jacobian_y(y, lo, hi), num, atol=1e-6)
    _, lq, _ = maf.forward(y, params)
    assert np.allclose(maf.log_q_theta(th, params, lo, hi), lq - num, atol=1e-6)


def test_gradient_matches_finite_differences(params):
    rng = np.random.default_rng(6)
    y = rng.normal(size=(64, 8))
    w = rng.uniform(0.1, 2.0, size=64)
    loss, grads = maf.loss_and_grad(y, w, params)
    M1, M2 = maf.masks(H_SMALL)
    masks = dict(W1=M1, W2=M2)
    for k in range(3):
        for key in ("W1", "b1", "W2", "b2"):
            shape = params[k][key].shape
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in shape)
                if key in masks and masks[key][idx] == 0:
                    assert grads[k][key][idx] == 0
                    continue
                old = params[k][key][idx]
                params[k][key][idx] = old + 1e-6
                lp, _ = maf.loss_and_grad(y, w, params)
                params[k][key][idx] = old - 1e-6
                lm, _ = maf.loss_and_grad(y, w, params)
                params[k][key][idx] = old
                num = (lp - lm) / 2e-6
                assert np.isclose(grads[k][key][idx], num, rtol=1e-5, atol=1e-8), (k, key, idx)


def test_adam_first_step_is_signed_learning_rate(params):
    """After one step m_hat / sqrt(v_hat) = g / |g|: every weight with a
    non-zero gradient moves by -lr sign(g) (up to eps)."""
    y = np.random.default_rng(7).normal(size=(32, 8))
    _, grads = maf.loss_and_grad(y, np.ones(32), params)
    before = [{k: v.copy() for k, v in p.items()} for p in params]
    maf.adam_step(params, grads, {}, lr=1e-2, eps=1e-12)
    for p0, p1, g in zip(before, params, grads):
        for key in p0:
            nz = np.abs(g[key]) > 1e-9
            assert np.allclose((p1[key] - p0[key])[nz], -1e-2 * np.sign(g[key][nz]), rtol=1e-6)
            assert np.all(p1[key][~nz] == p0[key][~nz]) or np.allclose(p1[key][~nz], p0[key][~nz], atol=1e-2)


def test_training_recovers_a_known_density():
    """y = A l + m with l iid standard logistic (A lower triangular): the flow
    can represent it exactly; its entropy is 8 * 2 + log |det A|."""
    rng = np.random.default_rng(8)
    A = np.tril(rng.normal(size=(8, 8)) * 0.3) + np.eye(8) * 0.7
    m = rng.normal(size=8)
    y = rng.logistic(size=(4000, 8)) @ A.T + m
    params = maf.init_params(rng, K=2, H=32, scale=0.3)
    state = {}
    for _ in range(1500):
        b = rng.integers(0, len(y), 256)
        _, g = maf.loss_and_grad(y[b], np.ones(256), params)
        maf.adam_step(params, g, state, lr=3e-3)
    u = rng.logistic(size=(20000, 8))
    ys, _ = maf.inverse(u, params)
    cov = (np.pi ** 2 / 3) * A @ A.T
    assert np.allclose(ys.mean(axis=0), m, atol=0.15)
    assert np.allclose(np.cov(ys.T), cov, atol=0.1 * np.abs(cov).max())
    # and the fitted density is close to the truth's entropy
    _, lq, _ = maf.forward(y, params)
    ent = 16.0 + np.linalg.slogdet(A)[1]
    assert abs(-lq.mean() - ent) < 0.1


def test_ess_fraction():
    assert maf.ess_fraction(np.ones(10)) == 1.0
    assert np.isclose(maf.ess_fraction(np.array([1.0, 0, 0, 0])), 0.25)


def test_bf16_rounding_is_round_to_nearest_even():
    import struct
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-9, 1.0 + 3 * 2**-9, -2.5, 1e-3, 3.14159265, 65504.0, 0.0])
    r = maf.round_bf16(vals)
    for v, got in zip(vals, r):
        b = struct.unpack("<I", struct.pack("<f", np.float32(v)))[0]
        lo, hi = b & 0xFFFF0000, (b & 0xFFFF0000) + 0x10000
        fl = [struct.unpack("<f", struct.pack("<I", x))[0] for x in (lo, hi)]
        d = [abs(np.float32(v) - f) for f in fl]
        want = fl[0] if d[0] < d[1] else fl[1] if d[1] < d[0] else fl[0 if ((lo >> 16) & 1) == 0 else 1]
        assert got == want, (v, got, want)


def test_flat_roundtrip(params):
    v = maf.flat(params)
    assert len(v) == 3 * (H_SMALL * 8 + H_SMALL + 16 * H_SMALL + 16)
    back = maf.unflat(v, 3, H_SMALL)
    for a, b in zip(params, back):
        for k in a:
            assert np.array_equal(a[k], b[k])


def test_edge_points_are_clamped_inside():
    y = maf.to_y(np.array([[0.0, 100.0, 1.0, 0.5, 0.5, 0.5, 0.5, 1.0]]), np.zeros(8),
                 np.array([1, 100, 2, 1, 1, 1, 1, 2.0]))
    assert np.all(np.isfinite(y))
    assert np.isclose(y[0, 0], np.log(2.0**-24) - np.log1p(-2.0**-24))


# --------------------------------------------------------------------------
# the bf16 mode of the backward pass (what the device's gradient is held to)
# --------------------------------------------------------------------------
def test_bf16_gradient_is_the_float64_gradient_with_rounded_operands(params, monkeypatch):
    """With the rounding made the identity, the bf16-mode backward pass is the
    float64 one (pinned against finite differences above) up to where the
    row weights are normalised; with rounding it stays within bfloat16's
    relative precision of it."""
    rng = np.random.default_rng(21)
    y = rng.normal(size=(300, 8))
    w = rng.uniform(0.2, 2.0, size=300)
    loss, grads, scales = maf.loss_and_grad(y, w, params, with_scale=True)
    lb, gb, sb = maf.loss_and_grad(y, w, params, bf16=True, with_scale=True)
    g, g_b = maf.flat(grads), maf.flat(gb)
    assert np.linalg.norm(g_b - g) < 1e-2 * np.linalg.norm(g) and abs(lb - loss) < 1e-2 * abs(loss)
    monkeypatch.setattr(maf, "round_bf16", lambda a: np.asarray(a, dtype=np.float64))
    li, gi, si = maf.loss_and_grad(y, w, params, bf16=True, with_scale=True)
    assert abs(li - loss) <= 1e-12 * abs(loss)
    assert np.allclose(maf.flat(gi), g, rtol=1e-10, atol=1e-14 * np.abs(g).max())
    assert np.allclose(maf.flat(si), maf.flat(scales), rtol=1e-10, atol=0)
    # the scale bounds the value: |sum of terms| <= sum of |terms|
    assert np.all(np.abs(g) <= maf.flat(scales) * (1 + 1e-12) + 1e-300)


def _device_like_gradient(y, w, params):
    """The gradient in the device's arithmetic, emulated on the CPU: float32
    everywhere, bfloat16 operands at every product, the row weights
    unnormalised until the end (an independent restatement of the backward
    pass, used to size the element-wise tolerance)."""
    f32 = np.float32

    def rb(a):
        return maf.round_bf16(a).astype(f32)

    H = params[0]["W1"].shape[0]
    M1, M2 = maf.masks(H)
    x, w = y.astype(f32), w.astype(f32)
    caches = []
    for p in params:
        W1, W2 = rb(p["W1"] * M1), rb(p["W2"] * M2)
        xb = rb(x)
        a1 = (xb @ W1.T).astype(f32) + p["b1"].astype(f32)
        hb = rb(np.maximum(a1, 0))
        out = (hb @ W2.T).astype(f32) + p["b2"].astype(f32)
        mu, al = out[:, :8], (6 * np.tanh(out[:, 8:] / 6)).astype(f32)
        z = ((x - mu) * np.exp(-al)).astype(f32)
        caches.append(dict(xb=xb, a1=a1, hb=hb, al=al, z=z, W1=W1, W2=W2))
        x = z[:, ::-1]
    gx = (w[:, None] * np.tanh(0.5 * x)).astype(f32)
    out = [None] * len(params)
    for k in reversed(range(len(params))):
        c = caches[k]
        gz = gx[:, ::-1]
        ex = np.exp(-c["al"]).astype(f32)
        r = c["al"] / f32(6)
        gout = np.concatenate([-gz * ex, (-gz * c["z"] + w[:, None]) * (f32(1) - r * r)], 1).astype(f32)
        gob = rb(gout)
        ga1 = rb(np.where(c["a1"] > 0, (gob @ c["W2"]).astype(f32), 0))
        out[k] = dict(W1=(ga1.T @ c["xb"]).astype(f32) * M1, b1=ga1.sum(0), W2=(gob.T @ c["hb"]).astype(f32) * M2,
                      b2=gout.sum(0))
        gx = (gz * ex + (ga1 @ c["W1"]).astype(f32)).astype(f32)
    return maf.flat(out).astype(np.float64) / float(w.sum())


@pytest.mark.parametrize("K,H,n", [(3, 64, 2000), (2, 208, 1500), (4, 256, 1100)])
def test_elementwise_gradient_bound_passes_device_arithmetic_and_fails_planted_mistakes(K, H, n):
    """The element-wise bound of tests/grad_check.py holds for the float32
    emulation of the device's arithmetic and fails for plausible mistakes:
    a sign on one block's db1, a factor of two on one 16-column group of one
    block's dW2 (one tensor-memory column group: 16 outputs x one 128-unit
    half), one input column of dW1 dropped, and the W1 gradients of two
    blocks exchanged."""
    from tests import grad_check
    rng = np.random.default_rng(K * 1000 + H)
    ps = maf.init_params(rng, K=K, H=H, scale=0.5)
    for p in ps:
        p["b1"] = rng.normal(0, 0.2, H)
        p["b2"] = rng.normal(0, 0.2, 16)
    ps = maf.unflat(maf.flat(ps).astype(np.float32).astype(np.float64), K, H)
    y = maf.to_y(rng.uniform(0.02, 0.98, size=(n, 8)), np.zeros(8), np.ones(8))
    w = rng.uniform(0.2, 2.0, size=n).astype(np.float32).astype(np.float64)
    _, gr, sc = maf.loss_and_grad(y, w, ps, bf16=True, with_scale=True)
    gref, scale = maf.flat(gr), maf.flat(sc)
    g = _device_like_gradient(y, w, ps)
    err, stray = grad_check.gradient_errors(g, gref, scale)
    assert stray == 0 and grad_check.gradient_close(g, gref, scale), grad_check.summary(err)
    # the layout of one block in the flat vector: W1 [H][8], b1 [H], W2 [16][H], b2 [16]
    size = 8 * H + H + 16 * H + 16

    def planted(fn):
        bad = [dict((key, v.copy()) for key, v in blk.items()) for blk in maf.unflat(g, K, H)]
        fn(bad)
        return maf.flat(bad)

    def flip_db1(b):
        b[0]["b1"] *= -1

    def double_w2_group(b):
        b[K - 1]["W2"][8:, :min(H, 128)] *= 2

    def drop_w1_column(b):
        b[0]["W1"][:, 3] = 0

    def swap_w1(b):
        if K > 1:
            b[0]["W1"], b[1]["W1"] = b[1]["W1"], b[0]["W1"]
        else:
            b[0]["W1"] = b[0]["W1"][::-1]

    for fn in (flip_db1, double_w2_group, drop_w1_column, swap_w1):
        bad = planted(fn)
        assert len(bad) == K * size
        assert not grad_check.gradient_close(bad, gref, scale), fn.__name__
