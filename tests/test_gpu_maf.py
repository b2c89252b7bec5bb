"""The flow proposal's BF16 tensor-core kernels against the float64 oracle.

Parity is checked against the oracle's bf16 mode, which rounds the inputs of
both matrix products (x, the hidden activations and the masked weights) to
bfloat16 exactly where the tensor-core products do; what remains is FP32
versus FP64 accumulation and elementwise math, plus the rare activation that
sits on a bfloat16 rounding boundary. Tolerances below are set from that:
typical |error| ~1e-5, bounded worst cases. Gradients are compared entry by
entry against the oracle's bf16-mode backward pass, each entry relative to
the sum of the absolute values of its terms (tests/grad_check.py)."""
import numpy as np
import pytest

from oracle import maf_oracle as mo
from tests import grad_check, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_14332_gb300 as abc  # noqa: E402
from paper_2012_14332_gb300 import build as _build  # noqa: E402

_build.build()
DEV = torch.device("cuda", 0)
LO = np.zeros(8)
HI = np.array([1, 100, 2, 1, 1, 1, 1, 2.0])


def _flow(K, H, seed, scale):
    params = mo.init_params(np.random.default_rng(seed), K=K, H=H, scale=scale)
    for p in params:
        p["b1"] = np.random.default_rng(seed + 1).normal(0, 0.2, p["b1"].shape)
        p["b2"] = np.random.default_rng(seed + 2).normal(0, 0.2, p["b2"].shape)
    v = mo.flat(params).astype(np.float32)
    f = abc.Flow(K, H)
    f.set_params(v)
    return f, mo.unflat(v.astype(np.float64), K, H)


def _thetas(n, seed):
    u = np.random.default_rng(seed).uniform(0.02, 0.98, size=(n, 8))
    return (LO + (HI - LO) * u).astype(np.float32)


@pytest.mark.parametrize("K,H", [(3, 256), (1, 16), (2, 64), (4, 128), (4, 256)])
def test_log_q_matches_oracle(K, H):
    f, params = _flow(K, H, 10 + K, 0.3)
    th = _thetas(5003, K)
    got = f.log_q(torch.from_numpy(th).to(DEV)).cpu().numpy().astype(np.float64)
    want = mo.log_q_theta(th.astype(np.float64), params, LO, HI, bf16=True)
    err = np.abs(got - want)
    print("log_q K=%d H=%d: median %.2e p99 %.2e max %.2e" % (K, H, np.median(err), np.quantile(err, 0.99), err.max()))
    assert np.median(err) < 1e-4 and np.quantile(err, 0.99) < 2e-3 and err.max() < 5e-2
    f.close()


@pytest.mark.parametrize("K,H", [(3, 256), (2, 32), (4, 256), (3, 144)])
def test_sample_matches_oracle_inverse(K, H):
    """The sampler is compiled per number of 16-unit chunks per degree: one
    (H = 32), two (H = 144) and three (H = 256)."""
    f, params = _flow(K, H, 20 + K, 0.3)
    n = 3001
    u = np.random.default_rng(3).logistic(size=(n, 8)).astype(np.float32)
    th, lq = f.sample(n, base=torch.from_numpy(u).to(DEV))
    th, lq = th.cpu().numpy().astype(np.float64), lq.cpu().numpy().astype(np.float64)
    y, lqy = mo.inverse(u.astype(np.float64), params, bf16=True)
    th_ref = mo.to_theta(y, LO, HI)
    lq_ref = lqy - mo.log_jacobian_y(y, LO, HI)
    rel = np.abs(th - th_ref) / (HI - LO)
    errq = np.abs(lq - lq_ref)
    print("sample K=%d H=%d: theta/width median %.2e p99 %.2e max %.2e; logq median %.2e p99 %.2e" % (
        K, H, np.median(rel), np.quantile(rel, 0.99), rel.max(), np.median(errq), np.quantile(errq, 0.99)))
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-3
    assert np.median(errq) < 1e-4 and np.quantile(errq, 0.99) < 5e-3
    # the density kernel agrees with the log-density the sampler reports
    lq2 = f.log_q(torch.from_numpy(th.astype(np.float32)).to(DEV)).cpu().numpy()
    inside = np.all((th_ref > LO + 1e-4 * (HI - LO)) & (th_ref < HI - 1e-4 * (HI - LO)), axis=1)
    ok = np.all(rel < 1e-3, axis=1) & inside
    assert np.median(np.abs(lq2[ok] - lq[ok])) < 1e-3
    f.close()


def test_zero_flow_draws_the_prior_from_the_documented_words():
    """A flow with zero parameters is the uniform prior: base coordinate c of
    sample j is logit(u), u = (2m + 1) 2^-24 from word c mod 4 of the Philox
    block with counter (i_lo, i_hi, 0, 4 stream + c / 4), i = first + j,
    key = seed (checked against the oracle's Philox). Each of the three blocks
    reverses the order, so theta_c = lo_c + w_c u_(7 - c); log q = -log volume."""
    import oracle
    f = abc.Flow(3, 256)
    n, seed, stream, first = 4096, 5, 3, (1 << 32) - 2000
    th, lq = f.sample(n, seed=seed, stream=stream, first_index=first)
    th = th.cpu().numpy().astype(np.float64)
    want = np.empty((n, 8))
    for j in range(n):
        i = first + j
        for g in range(2):
            w = oracle.philox4x32_10([i & 0xFFFFFFFF, i >> 32, 0, 4 * stream + g], [seed, 0])
            want[j, 4 * g:4 * g + 4] = ((w.astype(np.int64) & 0x7FFFFF) * 2 + 1) * 2.0 ** -24
    want = LO + (HI - LO) * want[:, ::-1]
    assert np.max(np.abs(th - want) / (HI - LO)) < 2e-6
    assert np.allclose(lq.cpu().numpy(), -np.log(np.prod(HI - LO)), atol=2e-4)
    big, _ = f.sample(1 << 18, seed=6)
    from scipy import stats
    u = (big.cpu().numpy().astype(np.float64) - LO) / (HI - LO)
    for c in range(8):
        assert stats.kstest(u[:, c], "uniform").pvalue > 1e-3, c
    f.close()


def _oracle_gradient(th, w, params):
    y = mo.to_y(th.astype(np.float64), LO, HI)
    loss, grads, scales = mo.loss_and_grad(y, w.astype(np.float64), params, bf16=True, with_scale=True)
    return loss, mo.flat(grads), mo.flat(scales)


def _check_elementwise(label, g, gref, scale):
    err, stray = grad_check.gradient_errors(g, gref, scale)
    med, p99, mx = grad_check.summary(err)
    worst = np.flatnonzero(scale > 0)[np.argmax(err)]
    print("%s: |g - g_ref| / scale median %.2e p99 %.2e max %.2e (entry %d: %.6e vs %.6e, scale %.3e); "
          "%d entries, %d with zero scale" % (label, med, p99, mx, worst, g[worst], gref[worst], scale[worst],
                                             len(err), int(np.count_nonzero(scale == 0))))
    assert stray == 0, "%d entries with no nonzero term are nonzero" % stray
    assert med <= grad_check.MEDIAN and p99 <= grad_check.P99 and mx <= grad_check.MAX, (med, p99, mx)


@pytest.mark.parametrize("K,H,n,scale", [(3, 64, 4096, 0.7), (2, 208, 3000, 0.7), (4, 256, 2069, 0.5),
                                         (1, 144, 1000, 0.7)])
def test_gradient_matches_oracle(K, H, n, scale):
    """The weight gradients accumulate in tensor memory per 128-unit half:
    H = 64 and 144 and 208 leave the last half partly filled (its padding
    lanes must be skipped), K = 4 x 256 uses all 256 allocated columns. Four
    blocks initialised at scale 0.7 compound their exp(-alpha) factors into a
    loss near 10^3 per point, where FP32 against FP64 differs by percents; at
    0.5 the loss is about 19, like the other shapes'. Every entry is compared
    with the oracle's bf16-mode gradient."""
    f, params = _flow(K, H, 31, scale)
    th = _thetas(n, 7)
    w = np.random.default_rng(8).uniform(0.2, 2.0, size=n).astype(np.float32)
    loss, g = f.gradient(torch.from_numpy(th).to(DEV), torch.from_numpy(w).to(DEV))
    loss_ref, gref, gscale = _oracle_gradient(th, w, params)
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    cos = g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref))
    print("gradient K=%d H=%d: loss %.6f vs %.6f, relative norm error %.3e, cosine %.9f" % (K, H, loss, loss_ref,
                                                                                           rel, cos))
    assert abs(loss - loss_ref) < 2e-3 * abs(loss_ref) + 1e-3
    _check_elementwise("gradient K=%d H=%d" % (K, H), g, gref, gscale)
    # masked entries have exactly zero gradient
    M1, M2 = mo.masks(H)
    zero = mo.flat([dict(W1=1 - M1, b1=np.zeros(H), W2=1 - M2, b2=np.zeros(16))] * K) > 0
    assert np.all(g[zero] == 0)
    # the whole vector as well
    assert rel < 1e-3 and cos > 0.999999
    f.close()


@pytest.mark.parametrize("K,H,n", [(3, 256, 2055), (3, 256, 2069), (2, 208, 2055)])
def test_wide_gradient_form_matches_the_narrow_one_and_the_oracle(K, H, n):
    """A set of 16 flows takes the wide (15 compute warps) gradient kernel,
    chosen when 4-warp CTAs would run more than two waves; flow 0's gradient
    there equals a one-flow object's (the 4-warp kernel) up to float summation
    order, and the oracle's bf16-mode gradient entry by entry. The point counts
    end in a partial tile; H = 208 leaves the second 128-unit half partly
    filled."""
    R = 16
    f1, params = _flow(K, H, 71, 0.5)
    fs = abc.Flow(K, H, n_flows=R)
    fs.set_params(np.stack([f1.get_params()] * R))
    th = _thetas(n, 5)
    w = np.random.default_rng(6).uniform(0.2, 2.0, size=n).astype(np.float32)
    thd, wd = torch.from_numpy(th).to(DEV), torch.from_numpy(w).to(DEV)
    loss_w, g_w = fs.gradient(thd, wd)
    loss_n, g_n = f1.gradient(thd, wd)
    rel = np.linalg.norm(g_w - g_n) / np.linalg.norm(g_n)
    print("wide vs narrow gradient (n=%d): loss %.7f vs %.7f, relative difference %.2e" % (n, loss_w, loss_n, rel))
    assert abs(loss_w - loss_n) < 1e-5 * abs(loss_n) and rel < 1e-4
    loss_ref, gref, gscale = _oracle_gradient(th, w, params)
    assert abs(loss_w - loss_ref) < 2e-3 * abs(loss_ref) + 1e-3
    _check_elementwise("wide gradient K=%d H=%d n=%d" % (K, H, n), g_w, gref, gscale)
    _check_elementwise("narrow gradient K=%d H=%d n=%d" % (K, H, n), g_n, gref, gscale)
    M1, M2 = mo.masks(H)
    zero = mo.flat([dict(W1=1 - M1, b1=np.zeros(H), W2=1 - M2, b2=np.zeros(16))] * K) > 0
    assert np.all(g_w[zero] == 0)
    f1.close()
    fs.close()


def test_gradient_wait_that_runs_out_reports_timeout_and_recovers():
    """The gradient kernel's waits are bounded. With the issuing thread held
    (no tensor-core products), its wait for them runs out after 2 s, the call
    returns ABC_ERR_TIMEOUT, and the next call on the same flow gives the
    same gradient as before. With many jobs per warp (3 blocks x 2 halves
    per tile, 4096 rows) a warp whose wait ran out skips its later waits, so
    the call still returns within about two wait limits (the jobs' wait and
    the CTA's final one), not one limit per job."""
    import time
    f, _ = _flow(1, 16, 41, 0.5)
    th = torch.from_numpy(_thetas(16, 3)).to(DEV)
    loss0, g0 = f.gradient(th)
    f.test_hold_products(True)
    with pytest.raises(abc.AbcError) as e:
        f.gradient(th)
    assert e.value.status == abc.binding.ABC_ERR_TIMEOUT
    f.test_hold_products(False)
    loss1, g1 = f.gradient(th)
    assert loss1 == loss0 and np.array_equal(g1, g0)
    f.close()
    f, _ = _flow(3, 256, 43, 0.5)
    th = torch.from_numpy(_thetas(4096, 4)).to(DEV)
    loss0, g0 = f.gradient(th)
    f.test_hold_products(True)
    t0 = time.monotonic()
    with pytest.raises(abc.AbcError) as e:
        f.gradient(th)
    took = time.monotonic() - t0
    print("held gradient over 4096 rows, 3 x 256: ABC_ERR_TIMEOUT after %.2f s" % took)
    assert e.value.status == abc.binding.ABC_ERR_TIMEOUT
    assert took < 7.0
    f.test_hold_products(False)
    loss1, g1 = f.gradient(th)
    assert loss1 == loss0 and np.array_equal(g1, g0)
    f.close()


def test_adam_step_matches_oracle():
    K, H = 2, 32
    f, params = _flow(K, H, 41, 0.5)
    th = _thetas(1000, 9)
    thd = torch.from_numpy(th).to(DEV)
    p0 = f.get_params().astype(np.float64)
    state = {}
    pv = mo.unflat(p0, K, H)
    for step in range(3):
        _, g = f.gradient(thd)
        f.adam_step(lr=1e-2)
        mo.adam_step(pv, mo.unflat(g.astype(np.float64), K, H), state, lr=1e-2)
    got = f.get_params().astype(np.float64)
    want = mo.flat(pv)
    assert np.max(np.abs(got - want)) < 1e-5
    f.close()


def test_training_fits_a_known_density():
    """Weighted maximum likelihood on the GPU: points y = A l + m in y = logit
    space (l iid standard logistic, A lower triangular, entropy
    16 + log |det A|) are fitted by a randomly initialised flow; the trained
    flow's cross-entropy approaches the truth's entropy and its samples match
    the truth's moments. The same data, initialisation scale and schedule
    trained by the float64 oracle reach the same loss."""
    rng = np.random.default_rng(12)
    A = np.tril(rng.normal(size=(8, 8)) * 0.3) + np.eye(8) * 0.6
    m = rng.normal(size=8) * 0.5
    y = rng.logistic(size=(20000, 8)) @ A.T + m
    th = mo.to_theta(y, LO, HI).astype(np.float32)
    ent = 16.0 + np.linalg.slogdet(A)[1]
    f = abc.Flow(3, 128)
    f.init_random(seed=3, scale=0.3)
    thd = torch.from_numpy(th).to(DEV)
    loss = f.train(thd, None, n_steps=1500, batch=1024, lr=2e-3, seed=1)
    # oracle: same data, same kind of initialisation and schedule
    params = mo.init_params(np.random.default_rng(3), K=3, H=128, scale=0.3)
    state = {}
    yy = mo.to_y(th.astype(np.float64), LO, HI)
    for _ in range(1500):
        b = rng.integers(0, len(yy), 1024)
        _, g = mo.loss_and_grad(yy[b], np.ones(1024), params)
        mo.adam_step(params, g, state, lr=2e-3)
    _, lq_o, _ = mo.forward(yy, params)
    print("train: GPU loss %.4f, oracle loss %.4f, truth entropy %.4f" % (loss, -lq_o.mean(), ent))
    assert loss < ent + 0.1
    assert abs(loss - (-lq_o.mean())) < 0.05
    ts, _ = f.sample(40000, seed=2)
    ys = mo.to_y(ts.cpu().numpy().astype(np.float64), LO, HI)
    cov = (np.pi ** 2 / 3) * A @ A.T
    assert np.allclose(ys.mean(0), m, atol=0.1)
    assert np.allclose(np.cov(ys.T), cov, atol=0.1 * np.abs(cov).max())
    f.close()


def test_flow_set_members_equal_single_flows():
    """Flow r of a set evaluates and samples exactly like a one-flow object
    holding the same parameters (the same kernels on flow r's copy)."""
    K, H, R = 3, 64, 3
    singles, vs = [], []
    for r in range(R):
        f, _ = _flow(K, H, 50 + r, 0.3)
        singles.append(f)
        vs.append(f.get_params())
    fs = abc.Flow(K, H, n_flows=R)
    fs.set_params(np.stack(vs))
    assert np.array_equal(fs.get_params(), np.stack(vs))
    th = torch.from_numpy(_thetas(1000, 3)).to(DEV)
    u = torch.from_numpy(np.random.default_rng(4).logistic(size=(777, 8)).astype(np.float32)).to(DEV)
    for r in range(R):
        assert torch.equal(fs.log_q(th, flow=r), singles[r].log_q(th))
        a, la = fs.sample(777, base=u, flow=r)
        b, lb = singles[r].sample(777, base=u)
        assert torch.equal(a, b) and torch.equal(la, lb)
        a, _ = fs.sample(2000, seed=9, stream=2, first_index=5, flow=r)
        b, _ = singles[r].sample(2000, seed=9, stream=2, first_index=5)
        assert torch.equal(a, b)
    with pytest.raises(abc.AbcError):
        fs.log_q(th, flow=R)
    for f in singles:
        f.close()
    fs.close()


@pytest.mark.parametrize("K,H,R", [(3, 256, 1), (2, 64, 1), (3, 112, 3), (4, 256, 2), (1, 208, 1)])
def test_training_steps_publish_what_a_full_publish_writes(K, H, R):
    """A training step's Adam launch republishes each parameter it updates, one
    thread per parameter, into every layout the kernels read (density,
    gradient and the sampler's degree-grouped copy), and training without
    validation ends on that. The densities, draws and gradient after training
    then equal those after a full republish of the same parameters, bit for
    bit: a parameter written to a wrong place, or not at all, would change
    them. Shapes: the paired and unpaired gradient forms, a set of flows, and
    one, two and three sampler chunks per degree."""
    fs = abc.Flow(K, H, n_flows=R)
    fs.init_random(seed=4, scale=0.3)
    p0 = fs.get_params().copy()
    data = [torch.from_numpy(_thetas(3000 + 500 * r, 30 + r)).to(DEV) for r in range(R)]
    fs.train_flows(data, None, n_steps=7, batch=512, lr=5e-3, seed=2)
    th = torch.from_numpy(_thetas(1500, 40)).to(DEV)

    def outputs():
        out = []
        for r in range(R):
            out.append(fs.log_q(th, flow=r).cpu().numpy())
            t, lq = fs.sample(999, seed=5, flow=r)
            out += [t.cpu().numpy(), lq.cpu().numpy()]
        loss, g = fs.gradient(th)
        return out + [np.array([loss]), g]

    p1 = fs.get_params()
    assert not np.array_equal(p1, p0)
    a = outputs()
    fs.set_params(p1)
    b = outputs()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    fs.close()


def test_train_flows_fits_each_flow_to_its_own_data():
    """One set trains three flows on three different densities (y = A l + m in
    y space, l iid standard logistic) in the same launches; each reaches its own
    data's entropy, and a flow given no data keeps its parameters bit for bit."""
    rng = np.random.default_rng(21)
    R = 4
    fs = abc.Flow(3, 128, n_flows=R)
    fs.init_random(seed=8, scale=0.3)
    p0 = fs.get_params().copy()
    data, ents, means = [], [], []
    for r in range(3):
        A = np.tril(rng.normal(size=(8, 8)) * 0.3) + np.eye(8) * (0.4 + 0.2 * r)
        m = rng.normal(size=8) * 0.5
        y = rng.logistic(size=(20000 + 5000 * r, 8)) @ A.T + m
        data.append(torch.from_numpy(mo.to_theta(y, LO, HI).astype(np.float32)).to(DEV))
        ents.append(16.0 + np.linalg.slogdet(A)[1])
        means.append(m)
    losses = fs.train_flows(data + [None], None, n_steps=1500, batch=1024, lr=2e-3, seed=1)
    p1 = fs.get_params()
    print("train_flows: losses %s, entropies %s" % (np.round(losses, 4), np.round(ents, 4)))
    for r in range(3):
        assert losses[r] < ents[r] + 0.1, r
        ts, _ = fs.sample(40000, seed=2, flow=r)
        ys = mo.to_y(ts.cpu().numpy().astype(np.float64), LO, HI)
        assert np.allclose(ys.mean(0), means[r], atol=0.15), r
    assert losses[3] == 0.0 and np.array_equal(p1[3], p0[3])
    assert not np.array_equal(p1[0], p0[0])
    fs.close()


def test_early_stopping_generalises_on_a_small_set():
    """300 points of a known Gaussian (y space): trained for up to 2000 steps,
    the flow that holds out 20 % and keeps its best validation parameters has a
    lower loss on fresh points of the same density than the flow trained on all
    300 to the end (which overfits them)."""
    rng = np.random.default_rng(33)
    A = np.tril(rng.normal(size=(8, 8)) * 0.3) + np.eye(8) * 0.5
    m = rng.normal(size=8) * 0.3
    small = mo.to_theta(rng.normal(size=(300, 8)) @ A.T + m, LO, HI).astype(np.float32)
    fresh = mo.to_theta(rng.normal(size=(50000, 8)) @ A.T + m, LO, HI).astype(np.float32)
    ent = 0.5 * np.linalg.slogdet(2 * np.pi * np.e * A @ A.T)[1]
    out = []
    for vf in (0.0, 0.2):
        f = abc.Flow(3, 128, n_flows=1)
        f.init_random(seed=4, scale=0.3)
        f.train_flows([torch.from_numpy(small).to(DEV)], None, n_steps=2000, batch=1024, lr=2e-3, seed=2,
                      val_fraction=vf)
        loss, _ = f.gradient(torch.from_numpy(fresh).to(DEV))
        out.append(loss)
        f.close()
    print("fresh-data loss: no validation %.4f, early stopping %.4f, entropy %.4f" % (out[0], out[1], ent))
    assert out[1] < out[0]


def test_broadened_proposal_matches_oracle():
    """With the base scaled by tau, sampling (given base draws) and the density
    follow the oracle's tau-broadened flow; tau = 1 is the trained flow."""
    K, H, tau = 3, 64, 1.4
    f, params = _flow(K, H, 61, 0.3)
    f.set_proposal_scale(tau)
    th = _thetas(3000, 11)
    got = f.log_q(torch.from_numpy(th).to(DEV)).cpu().numpy().astype(np.float64)
    want = mo.log_q_theta(th.astype(np.float64), params, LO, HI, bf16=True, tau=tau)
    err = np.abs(got - want)
    assert np.median(err) < 1e-4 and np.quantile(err, 0.99) < 2e-3
    u = np.random.default_rng(12).logistic(size=(2000, 8)).astype(np.float32)
    ts, lq = f.sample(2000, base=torch.from_numpy(u).to(DEV))
    y, lqy = mo.inverse(u.astype(np.float64), params, bf16=True, tau=tau)
    rel = np.abs(ts.cpu().numpy() - mo.to_theta(y, LO, HI)) / (HI - LO)
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-3
    assert np.median(np.abs(lq.cpu().numpy() - (lqy - mo.log_jacobian_y(y, LO, HI)))) < 1e-4
    with pytest.raises(abc.AbcError):
        f.set_proposal_scale(0.1)
    f.close()
