"""Learned tuner on the GPU against the oracle: features of the sampled
blocks (histogram fractions exact, other features within 1e-6), network
forward / gradient / Adam within 1e-4 of the oracle's double-precision
network, training that lowers the loss, and the tuning call's choices equal
to the argmax of the oracle's logits."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2310_14133_gb300 import build
    build.build()
    import paper_2310_14133_gb300 as q
    return q


def _field(shape, seed, slope=5.0 / 3.0):
    import synth
    return synth.grf(shape, slope, seed=seed, n_modes=96, device="cuda").contiguous()


CASES = [((100, 90, 110), 32, 0.005, 1e-3),    # one sampled block
         ((256, 256, 256), 32, 0.005, 1e-4),   # eight blocks
         ((20, 30, 40), 32, 0.005, 1e-2),      # no block fits: the whole field
         ((37, 300, 29), 16, 0.005, 1e-3),     # blocks along one axis, whole extent on others
         ((300, 517), 64, 0.01, 1e-3),         # 2-D, one block
         ((1800, 3600), 64, 0.01, 1e-3)]       # 2-D, 18 blocks


@pytest.mark.parametrize("shape,block,rate,rel", CASES)
def test_features_parity(q, orc, shape, block, rate, rel):
    x = _field(shape, seed=sum(shape))
    opts = q.make_tune_opts(block=block, rate=rate)
    f = q.features(x, rel, opts)
    xn = x.cpu().numpy()
    mn, mx, _ = orc.value_range(xn)
    ref = orc.features(xn, rel, float(mx) - float(mn), block, rate)
    assert np.array_equal(f[10:58], ref[10:58]), "histogram fractions"
    # sums of many terms: compensated binary32 per thread against double
    np.testing.assert_allclose(f[:10], ref[:10], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(f[58:], ref[58:], rtol=1e-6, atol=1e-9)
    # the device copy is the same values in binary32
    d = torch.empty(64, dtype=torch.float32, device="cuda")
    q.features(x, rel, opts, device_out=d)
    assert np.array_equal(d.cpu().numpy(), f.astype(np.float32))


def _net(seed):
    rng = np.random.default_rng(seed)
    P = (rng.normal(0, 1, 26896) * 0.15).astype(np.float32)
    mean = rng.normal(0, 1, 64).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, 64).astype(np.float32)
    sd[7] = 0.0
    return P, mean, sd


def _data(seed, B):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 2, (B, 64)).astype(np.float32)
    lab = np.stack([rng.integers(0, n, B) for n in (2, 6, 5, 3)], axis=1).astype(np.int32)
    return X, lab


def _close(a, b, rel=1e-4):
    scale = max(1e-30, float(np.abs(b).max()))
    err = np.abs(a.astype(np.float64) - b)
    assert np.all(err <= rel * np.abs(b) + 1e-5 * scale), float((err / scale).max())


@pytest.mark.parametrize("B", [1, 16, 37])
def test_network_forward_gradient_parity(q, orc, B):
    P, mean, sd = _net(B)
    X, lab = _data(100 + B, B)
    m = q.Model(seed=1)
    m.set(P, mean, sd)
    Xd = torch.from_numpy(X).cuda()
    labd = torch.from_numpy(lab).cuda()
    logits = m.forward(Xd).cpu().numpy()
    P64, mean64, sd64 = P.astype(np.float64), mean.astype(np.float64), sd.astype(np.float64)
    ref = orc.mlp_forward(P64, mean64, sd64, X.astype(np.float64))
    _close(logits, ref)
    loss, g = m.gradient(Xd, labd)
    rloss, rg = orc.mlp_loss_grad(P64, mean64, sd64, X.astype(np.float64), lab)
    assert loss == pytest.approx(rloss, rel=1e-5)
    _close(g.cpu().numpy(), rg)
    # the gradient call leaves the weights alone
    assert np.array_equal(m.get()[0], P)
    m.free()


def test_adam_step_parity(q, orc):
    P, mean, sd = _net(5)
    X, lab = _data(6, 40)
    m = q.Model(seed=2)
    m.set(P, mean, sd)
    Xd, labd = torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda()
    P64 = P.astype(np.float64)
    mm, vv = np.zeros_like(P64), np.zeros_like(P64)
    for t in (1, 2, 3):
        _, rg = orc.mlp_loss_grad(P64, mean.astype(np.float64), sd.astype(np.float64),
                                  X.astype(np.float64), lab)
        orc.adam_step(P64, rg, mm, vv, t, lr=1e-3)
        m.train_step(Xd, labd, 1e-3)
        got = m.get()[0].astype(np.float64)
        # an Adam step moves a parameter by at most lr (1 - b1) / sqrt(1 - b2);
        # parameters with a clear gradient move the same way on both sides
        assert np.abs(got - P.astype(np.float64)).max() <= t * 3.2e-3
        big = np.abs(rg) > 1e-3 * np.abs(rg).max()
        np.testing.assert_allclose(got[big], P64[big], rtol=0, atol=2e-5 * t)
    m.free()


def test_training_lowers_loss(q):
    rng = np.random.default_rng(9)
    B = 512
    X = rng.normal(0, 1, (B, 64)).astype(np.float32)
    W = rng.normal(0, 1, (64, 16))
    z = X @ W
    lab = np.stack([np.argmax(z[:, o:o + n], axis=1) for o, n in ((0, 2), (2, 6), (8, 5),
                                                                  (13, 3))], 1).astype(np.int32)
    m = q.Model(seed=3)
    Xd, labd = torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda()
    first = m.train_step(Xd, labd, 3e-3, want_loss=True)
    for _ in range(300):
        last = m.train_step(Xd, labd, 3e-3, want_loss=True)
    assert last < 0.3 * first, (first, last)
    m.free()


@pytest.mark.parametrize("shape", [(96, 100, 120), (400, 700)])
def test_tune_learned_follows_network(q, orc, shape):
    x = _field(shape, seed=7)
    P, mean, sd = _net(11)
    m = q.Model()
    m.set(P, mean, sd)
    nd = len(shape)
    block, rate = (32, 0.005) if nd == 3 else (64, 0.01)
    opts = q.make_tune_opts(block=block, rate=rate, alphas=[1.0, 1.25, 1.5, 1.75, 2.0],
                            betas=[2.0, 3.0, 4.0])
    rep = q.tune_learned(x, 1e-3, m, opts=opts)
    xn = x.cpu().numpy()
    mn, mx, _ = orc.value_range(xn)
    vr = float(mx) - float(mn)
    f = orc.features(xn, 1e-3, vr, block, rate)
    lo = orc.mlp_forward(P.astype(np.float64), mean.astype(np.float64), sd.astype(np.float64),
                         f.astype(np.float32).astype(np.float64))[0]
    want = []
    for off, n in ((0, 2), (2, 6 if nd == 3 else 2), (8, 5), (13, 3)):
        z = lo[off:off + n]
        top = np.sort(z)[::-1]
        assert top[0] - top[1] > 1e-3, "near-tie: choose another seed"
        want.append(int(np.argmax(z)))
    assert rep.params.interp[0] == want[0] and rep.params.order[0] == want[1]
    assert rep.params.alpha == [1.0, 1.25, 1.5, 1.75, 2.0][want[2]]
    assert rep.params.beta == [2.0, 3.0, 4.0][want[3]]
    assert rep.abs_eb == 1e-3 * vr and rep.n_trials == 0
    # PSNR target: the uniform-error estimate when it is below the bound
    rep2 = q.tune_learned(x, 1e-2, m, metric=q.METRIC_PSNR, target=80.0, opts=opts)
    assert rep2.abs_eb == pytest.approx(vr * math.sqrt(3) * 10 ** (-4.0), rel=1e-12)
    m.free()


def test_label_collection_resumes_from_cache(q, tmp_path):
    # an interrupted collection (3 of 5 samples) resumes from its cache and
    # gives the rows a fresh collection gives
    from paper_2310_14133_gb300 import learn
    opts = q.make_tune_opts(block=16, rate=0.05, n_orders=2, alphas=[1.0, 1.5, 2.0],
                            betas=[2.0, 4.0])
    samples = [(_field((40, 40, 40), 50 + i), 1e-3) for i in range(5)]
    cache = str(tmp_path / "labels.npz")
    X3, Y3 = learn.collect(samples[:3], opts, cache=cache)
    assert X3.shape == (3, q.NFEATURES) and Y3.shape == (3, 4)
    X5, Y5 = learn.collect(samples, opts, cache=cache)
    Xf, Yf = learn.collect(samples, opts)
    assert torch.equal(Y5, Yf) and torch.equal(X5, Xf)
    d = np.load(cache)
    assert d["features"].shape == (5, q.NFEATURES) and d["labels"].shape == (5, 4)


def test_tune_learned_verified_against_oracle(q, orc):
    """The network proposes the setting (one interpolator and order for every
    level, alpha, beta) and the sampled trials verify it in the PSNR-target
    mode: its bound, rate and metric follow the oracle's target-mode steps on
    that setting (trials at e0 and at 1.2 e0 or 0.8 e0, the secant on log e,
    the final pick), and the setting is the network's."""
    x = _field((96, 100, 120), seed=7)
    P, mean, sd = _net(11)
    m = q.Model()
    m.set(P, mean, sd)
    alphas, betas = [1.0, 1.25, 1.5, 1.75, 2.0], [2.0, 3.0, 4.0]
    opts = q.make_tune_opts(block=16, rate=0.05, alphas=alphas, betas=betas)
    target = 70.0
    prop = q.tune_learned(x, 1e-2, m, opts=opts)
    rep = q.tune_learned_verified(x, 1e-2, m, metric=q.METRIC_PSNR, target=target, opts=opts)
    assert list(rep.params.interp[:5]) == list(prop.params.interp[:5])
    assert list(rep.params.order[:5]) == list(prop.params.order[:5])
    assert (rep.params.alpha, rep.params.beta) == (prop.params.alpha, prop.params.beta)
    xn = x.cpu().numpy()
    mn, mx, _ = orc.value_range(xn)
    vr = float(mx) - float(mn)
    org, bd, _ = orc.sample_blocks(xn.shape, 16, 0.05)
    assert org.shape[0] > 1
    op = orc.make_params(3, interp=int(prop.params.interp[0]), order=int(prop.params.order[0]),
                         alpha=prop.params.alpha, beta=prop.params.beta, anchor_stride=16)
    e_user = 1e-2 * vr
    e0 = min(vr * math.sqrt(3.0) * 10.0 ** (-target / 20.0), e_user)

    def trial(e):
        t = orc.block_trial(xn, org, bd, op, e, vrange=vr)
        return e, t.B, orc.trial_metric(t, orc.METRIC_PSNR, vr)

    pts = [trial(e0)]
    pts.append(trial(orc.target_scale(pts[0][2], target) * e0))
    for _ in range(4):
        en = orc.secant_step(pts[-2][0], pts[-2][2], pts[-1][0], pts[-1][2], target, e0, e_user)
        if en is None:
            break
        pts.append(trial(en))
    k = orc.target_pick([p[0] for p in pts], [p[2] for p in pts], target, e_user)
    assert rep.abs_eb == pytest.approx(pts[k][0], rel=1e-5)
    assert rep.B == pytest.approx(pts[k][1], rel=1e-5)
    assert rep.M == pytest.approx(pts[k][2], rel=1e-6)
    assert rep.M >= target
    m.free()


def _stretched_field(n, axis, stretch, slope, seed, modes=64):
    """A Gaussian random field whose wavenumbers along `axis` are divided by
    `stretch`: smooth along that axis, rough along the others (test input:
    the recipe's random Fourier modes with one axis stretched)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    d = torch.randn(modes, 3, generator=g, dtype=torch.float64)
    d = d / d.norm(dim=1, keepdim=True)
    kmag = torch.exp(torch.rand(modes, generator=g, dtype=torch.float64) * math.log(n / 4.0))
    k = d * kmag[:, None]
    k[:, axis] /= stretch
    amp = kmag ** ((1.0 - slope) / 2.0)
    phase = torch.rand(modes, generator=g, dtype=torch.float64) * 2.0 * math.pi
    c = torch.arange(n, dtype=torch.float64, device="cuda") / n
    f = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    for m in range(modes):
        arg = (2.0 * math.pi * (k[m, 0] * c[:, None, None] + k[m, 1] * c[None, :, None]
                                + k[m, 2] * c[None, None, :]) + phase[m])
        f += amp[m] * torch.cos(arg)
    f *= 3.0 / f.std()
    return f.float().contiguous()


def test_trained_network_gains_over_default_setting(q):
    """What the trained network gains: labelled by the sampled tuner on a few
    hundred small fields, each smooth along a random axis, the network picks
    for a held-out field that is smooth along z a setting that compresses it
    better than the fixed default (cubic, dimension order z, y, x,
    alpha = beta = 1), at the same bound."""
    from paper_2310_14133_gb300 import learn
    opts = q.make_tune_opts(block=16, rate=0.05, alphas=[1.0, 1.25, 1.5, 1.75, 2.0],
                            betas=[2.0, 3.0, 4.0])
    rng = np.random.default_rng(3)

    def samples():
        for i in range(240):
            axis = int(rng.integers(0, 3))
            stretch = float(rng.choice([1.0, 4.0, 8.0]))
            slope = float(rng.uniform(1.5, 3.0))
            rel = float(10.0 ** rng.uniform(-4.0, -2.0))
            yield _stretched_field(48, axis, stretch, slope, 1000 + i), rel

    X, Y = learn.collect(samples(), opts)
    m = q.Model(seed=4)
    learn.fit(m, X, Y, epochs=200, batch=64, lr=3e-3)
    x = _stretched_field(96, 0, 8.0, 2.0, 77)
    rel = 1e-3
    rl = q.tune_learned(x, rel, m, opts=opts)
    crs = {}
    for name, p in (("learned", rl.params), ("default", q.make_params(3))):
        b = q.compress_abs(x, rl.abs_eb, p)
        crs[name] = b.info().est_ratio
        b.free()
    assert crs["learned"] > 1.02 * crs["default"], crs
    m.free()
