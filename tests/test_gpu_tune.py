"""GPU sampled tuner (Sec. 6) against the oracle's tuner on the same fields:
the chosen interpolators, orders, alpha and beta must be identical; the
sampled bit rate is exact (integer histograms).  The Algorithm 1 scores and
the sampled metrics are sums of many terms that the GPU accumulates in
compensated binary32 per thread (double arithmetic is slow on this part)
and the oracle in double, so they agree to 1e-6 relative, the metric
tolerance of the whole path."""

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


def _field(n=64, seed=21, nd=3):
    import synth
    if nd == 3:
        f = synth.grf((n, n, n), 5.0 / 3.0, seed=seed, n_modes=128).numpy()
        f += synth.fronts((n, n, n), 2000, count=4).numpy()
    else:
        f = (synth.zonal_bands(n, 2 * n, seed) + synth.grf((n, 2 * n), 3.0, seed=seed,
                                                          sigma=1.0)).numpy()
    return f


def _compare(q, orc, x, rel, metric, target, block, rate, n_orders, alphas, betas, m_rel=1e-6):
    xd = torch.from_numpy(x).cuda()
    qo = q.make_tune_opts(block=block, rate=rate, n_orders=n_orders, alphas=alphas, betas=betas)
    rep = q.tune(xd, rel, metric, target, qo)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    oo = orc.make_tune_opts(x.ndim, block=block, rate=rate, n_orders=n_orders, alphas=alphas,
                            betas=betas)
    ref = orc.tune(x, rel * vr, vr, metric, target, oo)
    L = int(math.log2(ref.params.anchor_stride))
    assert list(rep.params.interp[:L]) == list(ref.params.interp[:L])
    assert list(rep.params.order[:L]) == list(ref.params.order[:L])
    assert (rep.params.alpha, rep.params.beta) == (ref.params.alpha, ref.params.beta)
    assert rep.n_blocks == ref.n_blocks and rep.n_sampled_points == ref.n_sampled_points
    for l in range(L):
        assert rep.alg1_score[l] == pytest.approx(ref.alg1_score[l], rel=1e-6, abs=0)
    # the target mode's secant runs on the sampled metric: bound to 1e-5
    assert rep.abs_eb == pytest.approx(ref.e, rel=1e-5)
    assert rep.B == pytest.approx(ref.B, rel=1e-5)
    if metric != 0:
        assert rep.M == pytest.approx(ref.M, rel=m_rel)
    return rep, ref


@pytest.mark.parametrize("n_orders", [2, 6])
def test_bound_mode(q, orc, n_orders):
    x = _field(64, 21)
    rep, ref = _compare(q, orc, x, 1e-3, 0, float("nan"), 16, 0.05, n_orders,
                        [1.0, 1.25, 1.5, 1.75, 2.0], [2.0, 3.0, 4.0])
    assert rep.B == ref.B           # exact: pooled histograms are integers


def test_psnr_table1_mode(q, orc):
    x = _field(64, 22)
    _compare(q, orc, x, 1e-3, 1, float("nan"), 16, 0.05, 2, None, None)


def test_ssim_table1_mode(q, orc):
    x = _field(48, 23)
    _compare(q, orc, x, 1e-2, 2, float("nan"), 16, 0.2, 2, [1.0, 1.5, 2.0], [2.0, 4.0])


@pytest.mark.parametrize("target", [60.0, 80.0])
def test_psnr_target_mode(q, orc, target):
    x = _field(64, 24)
    rep, ref = _compare(q, orc, x, 1e-2, 1, target, 16, 0.05, 2, None, None)
    assert rep.M >= target


def test_ssim_target_mode(q, orc):
    x = _field(48, 25)
    _compare(q, orc, x, 2e-2, 2, 0.99, 16, 0.2, 2, [1.0, 1.5, 2.0], [2.0, 4.0])


def test_2d_bound_mode(q, orc):
    x = _field(300, 26, nd=2)
    _compare(q, orc, x, 1e-3, 0, float("nan"), 64, 0.05, 2, None, None)


def test_full_size_512_sampled_tuner(q, orc):
    """The plain-method-at-scale workload: 512^3 field with fronts, 0.5 %
    sampled 33^3 blocks, 12 interpolators, alpha 5 x beta 3, max-CR mode."""
    import synth
    xg = synth.grf_fronts_field(512, device="cuda")
    x = xg.cpu().numpy()
    del xg
    rep, ref = _compare(q, orc, x, 1e-3, 0, float("nan"), 32, 0.005, 6,
                        [1.0, 1.25, 1.5, 1.75, 2.0], [2.0, 3.0, 4.0])
    assert rep.n_blocks == 27


@pytest.mark.parametrize("metric,target", [(1, 70.0), (2, 0.9995)])
def test_verify_reproduces_target_mode(q, orc, metric, target):
    """Sampled verification of the setting the target mode chose runs the same
    trials (e0, then 0.8 e0 or 1.2 e0, then the secant), so it reproduces the
    tuner's bound, rate and metric exactly."""
    x = _field(64, seed=31)
    xd = torch.from_numpy(x).cuda()
    qo = q.make_tune_opts(block=16, rate=0.05)
    rep = q.tune(xd, 1e-2, metric, target, qo)
    ver = q.tune_verify(xd, 1e-2, rep.params, metric, target, qo)
    assert ver.abs_eb == rep.abs_eb and ver.B == rep.B and ver.M == rep.M
    assert list(ver.params.interp) == list(rep.params.interp)


def test_verify_fixed_bound_matches_oracle_trial(q, orc):
    x = _field(64, seed=32)
    xd = torch.from_numpy(x).cuda()
    qo = q.make_tune_opts(block=16, rate=0.05)
    p = q.make_params(3, interp=[1, 0, 1, 1, 0], order=[2, 5, 0, 1, 3], alpha=1.5, beta=3.0)
    ver = q.tune_verify(xd, 1e-3, p, q.METRIC_PSNR, float("nan"), qo)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    org, bd, _ = orc.sample_blocks(x.shape, 16, 0.05)
    op = orc.make_params(3, interp=[1, 0, 1, 1, 0], order=[2, 5, 0, 1, 3], alpha=1.5, beta=3.0,
                         anchor_stride=16)
    t = orc.block_trial(x, org, bd, op, 1e-3 * vr, vrange=vr)
    assert ver.abs_eb == 1e-3 * vr and ver.n_trials == 1
    assert ver.B == pytest.approx(t.B, rel=1e-12)
    assert ver.M == pytest.approx(orc.trial_metric(t, 1, vr), rel=1e-6)


def test_ac_table1_mode(q, orc):
    # AC-preferred mode: M = -AC (lag 1, pooled over the blocks), Table I with
    # the 0.8 e / 1.2 e trials
    x = _field(64, 24)
    rep, ref = _compare(q, orc, x, 1e-3, 3, float("nan"), 16, 0.05, 2,
                        [1.0, 1.25, 1.5, 1.75, 2.0], [2.0, 3.0, 4.0], m_rel=1e-5)
    assert -1.0 <= rep.M <= 1.0


def test_ac_target_is_rejected(q):
    x = torch.from_numpy(_field(32, 25)).cuda()
    with pytest.raises(q.QozError):
        q.tune(x, 1e-3, q.METRIC_AC, 0.1, q.make_tune_opts())


def test_bound_mode_many_codes(q, orc):
    # a tiny bound on a noisy field: thousands of distinct codes per trial
    # histogram, so the prefix-code cost runs on runs of equal counts and the
    # large counts' sort; the sampled bit rate must still be exact
    rng = np.random.default_rng(7)
    x = _field(48, 26) + rng.standard_normal((48, 48, 48)).astype(np.float32)
    rep, ref = _compare(q, orc, x, 1e-5, 0, float("nan"), 16, 0.3, 2,
                        [1.0, 1.5, 2.0], [2.0, 4.0])
    assert rep.B == ref.B
