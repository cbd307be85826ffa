"""Pins for the oracle's online tuner (Sec. 6): uniform block sampling
(Sec. 6.1), Algorithm 1 (Sec. 6.2), the alpha/beta candidates (Sec. 6.3.1)
and the Table I comparisons (Sec. 6.3.2)."""

import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_sampling_stride_paper_example(orc):
    # Sec. 6.1: 4x4 blocks on stride 10 sample 16 % of a 2D field
    org, bd, S = orc.sample_blocks((100, 100), 4, 0.16)
    assert S == 10
    assert org.shape[0] == 10 * 10


@pytest.mark.parametrize("shape,b,r,S,nb", [
    ((512, 512, 512), 32, 0.005, 187, 27),
    ((1024, 1024, 1024), 32, 0.005, 187, 216),
    ((1800, 3600), 64, 0.01, 640, 18),
    ((512, 512, 512), 16, 0.005, 94, 216),
])
def test_sampling_counts(orc, shape, b, r, S, nb):
    org, bd, s = orc.sample_blocks(shape, b, r)
    assert s == S
    assert org.shape[0] == nb
    assert bd == tuple([b + 1] * len(shape))
    nd = len(shape)
    assert np.all(org[:, :nd] + b <= np.array(shape) - 1)      # blocks lie inside
    assert np.all(org[:, :nd] % S == 0)                          # on the stride grid


def test_sampling_small_field_falls_back_to_full_extent(orc):
    org, bd, S = orc.sample_blocks((10, 100, 100), 16, 0.005)
    assert bd == (10, 17, 17)
    assert np.all(org[:, 0] == 0)


def test_table1_golden(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_cases.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for b1, m1, b2, m2, b2p, m2p, scale, dec in rows:
        b1, m1, b2, m2 = map(float, (b1, m1, b2, m2))
        d, sc = orc.table1(b1, m1, b2, m2)
        if float(scale) == 0:
            assert d == int(dec)
        else:
            assert d == -1 and sc == pytest.approx(float(scale))
            d2, _ = orc.table1(b1, m1, b2, m2, float(b2p), float(m2p))
            assert d2 == int(dec)


def _field(n=48, seed=7):
    import synth
    f = synth.grf((n, n, n), 5.0 / 3.0, seed=seed, n_modes=128).numpy()
    f += synth.fronts((n, n, n), 2000, count=3).numpy()
    return f


def test_alg1_inherits_top_sampled_level(orc):
    # Algorithm 1: L = log2 min(b, s); with b = 16 < s = 32 the full field's
    # level 5 reuses the choice made on level 4 (Sec. 6.2)
    x = _field()
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    o = orc.make_tune_opts(3, block=16, rate=0.05)
    r = orc.tune(x, 1e-3 * vr, vr, orc.METRIC_MAXERR, opts=o)
    assert r.params.interp[4] == r.params.interp[3]
    assert r.params.order[4] == r.params.order[3]
    assert r.alg1_score[4] == 0.0 and r.alg1_score[3] > 0.0


def _candidates(nd, n_orders):
    orders = [0, 1] if nd == 2 else ([0, 1, 2, 3, 4, 5] if n_orders == 6 else [0, 5])
    return [(t, o) for t in (0, 1) for o in orders]


@pytest.mark.parametrize("n_orders", [2, 6])
def test_alg1_and_bound_mode_brute_force(orc, n_orders):
    """Every level's interpolator minimises the mean L1 among all candidates
    given the levels above (Algorithm 1); (alpha, beta) minimises the sampled
    bit rate over the whole candidate grid in the max-CR mode (Sec. 7.2.2)."""
    x = _field(40, seed=9)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    e = 1e-3 * vr
    o = orc.make_tune_opts(3, block=16, rate=0.08, n_orders=n_orders, betas=[2.0, 3.0, 4.0])
    r = orc.tune(x, e, vr, orc.METRIC_MAXERR, opts=o)
    org, bd, _ = orc.sample_blocks(x.shape, 16, 0.08)
    cands = _candidates(3, n_orders)
    chosen = orc.make_params(3, anchor_stride=16)
    for l in (4, 3, 2, 1):
        scores = []
        for t, od in cands:
            p = orc.make_params(3, anchor_stride=16)
            for ll in range(l + 1, 5):
                p.interp[ll - 1] = chosen.interp[ll - 1]
                p.order[ll - 1] = chosen.order[ll - 1]
            p.interp[l - 1], p.order[l - 1] = t, od
            tr = orc.block_trial(x, org, bd, p, e, stop_level=l)
            scores.append(tr.stats.l1[l - 1] / tr.stats.cnt[l - 1])
        best = int(np.argmin(scores))
        # the oracle's choice is the first candidate within 1e-12 of the minimum
        first = next(i for i, s in enumerate(scores) if s <= scores[best] * (1 + 1e-12))
        assert (r.params.interp[l - 1], r.params.order[l - 1]) == cands[first]
        chosen.interp[l - 1], chosen.order[l - 1] = cands[first]
    bs = []
    for a in [1.0, 1.25, 1.5, 1.75, 2.0]:
        for b in [2.0, 3.0, 4.0]:
            p = orc.make_params(3, anchor_stride=16, alpha=a, beta=b)
            for ll in range(4):
                p.interp[ll], p.order[ll] = chosen.interp[ll], chosen.order[ll]
            bs.append((orc.block_trial(x, org, bd, p, e).B, a, b))
    bmin = min(v[0] for v in bs)
    first = next(v for v in bs if v[0] == bmin)
    assert (r.params.alpha, r.params.beta) == (first[1], first[2])
    assert r.B == bmin
    assert r.e == e


def test_fixed_bound_psnr_mode_runs_table1(orc):
    x = _field(40, seed=11)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    o = orc.make_tune_opts(3, block=16, rate=0.08)
    r = orc.tune(x, 1e-3 * vr, vr, orc.METRIC_PSNR, opts=o)
    # 4 levels x 4 candidates + 20 alpha/beta trials + extra Table I trials
    assert r.n_trials >= 16 + 20
    assert r.params.alpha in (1.0, 1.25, 1.5, 1.75, 2.0)
    assert r.params.beta in (1.5, 2.0, 3.0, 4.0)
    assert r.e == 1e-3 * vr


def test_target_psnr_mode_meets_target_on_samples(orc):
    x = _field(40, seed=13)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    o = orc.make_tune_opts(3, block=16, rate=0.08)
    for target in (60.0, 80.0):
        r = orc.tune(x, 1e-2 * vr, vr, orc.METRIC_PSNR, target=target, opts=o)
        assert r.M >= target
        assert r.e <= 1e-2 * vr
        # uniform-error start e0 = vr sqrt(3) 10^(-P/20) is within a factor 4
        e0 = vr * math.sqrt(3) * 10 ** (-target / 20)
        assert e0 / 16 <= r.e <= e0 * 4


def test_ac_mode(orc):
    """The AC-preferred mode (Sec. 7.2.2's autocorrelation mode): Table I with
    M = -AC; the reported metric is the chosen setting's pooled lag-1 AC over
    the sampled blocks, recomputed here from the error blocks themselves."""
    x = _field(40, seed=17)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    e = 1e-3 * vr
    o = orc.make_tune_opts(3, block=16, rate=0.08, betas=[2.0, 3.0, 4.0])
    r = orc.tune(x, e, vr, orc.METRIC_AC, opts=o)
    assert r.n_trials >= 16 + 15
    org, bd, _ = orc.sample_blocks(x.shape, 16, 0.08)
    p = orc.make_params(3, anchor_stride=16, alpha=r.params.alpha, beta=r.params.beta)
    for ll in range(4):
        p.interp[ll], p.order[ll] = r.params.interp[ll], r.params.order[ll]
    t = orc.block_trial(x, org, bd, p, e)
    assert r.M == pytest.approx(orc.trial_metric(t, orc.METRIC_AC, vr), abs=0, rel=1e-15)
    # the trial's AC is the pinned block-pooled definition applied to the
    # blocks' own compression errors
    errs, sizes = [], []
    for o3 in org:
        blk = np.ascontiguousarray(x[o3[0]:o3[0] + bd[0], o3[1]:o3[1] + bd[1],
                                     o3[2]:o3[2] + bd[2]])
        rec = orc.compress(blk, e, p)["recon"]
        errs.append((rec.astype(np.float64) - blk.astype(np.float64)).ravel())
        sizes.append(blk.size)
    assert t.ac == pytest.approx(orc.autocorr_blocks(np.concatenate(errs), sizes, 1), abs=1e-15)
    assert -1.0 <= r.M <= 1.0
    with pytest.raises(ValueError):
        orc.tune(x, e, vr, orc.METRIC_AC, target=0.1, opts=o)
