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


# ---- the tuner's selection rules on hand-worked numbers (Sec. 6.3.2, Table I)

class _Retrials:
    """Second points of solution II, keyed by (candidate, scale); every call
    is recorded so that a test can require exactly the calls Table I asks for."""

    def __init__(self, table):
        self.table = table
        self.calls = []

    def __call__(self, k, scale):
        key = (k, round(scale, 6))
        self.calls.append(key)
        return self.table[key]


def test_select_fixed_case3_keeps_incumbent_above_line(orc):
    # I = (2.5, 57) incumbent, II = (2.0, 50): B_I > B_II and M_I > M_II is
    # case 3, so II runs again at 0.8 e and lands at (3.0, 60); the line
    # through II's two points is 55 at B_I = 2.5 and M_I = 57 lies above it.
    rt = _Retrials({(1, 0.8): (3.0, 60.0)})
    assert orc.select_fixed([2.5, 2.0], [57.0, 50.0], retrial=rt) == 0
    assert rt.calls == [(1, 0.8)]


def test_select_fixed_case4_challenger_replaces_below_line(orc):
    # I = (2.5, 55), II = (3.0, 60): case 4, II again at 1.2 e -> (2.0, 52);
    # the line is 56 at B_I = 2.5 and M_I = 55 lies below it: II is kept.
    rt = _Retrials({(1, 1.2): (2.0, 52.0)})
    assert orc.select_fixed([2.5, 3.0], [55.0, 60.0], retrial=rt) == 1
    assert rt.calls == [(1, 1.2)]


def test_select_fixed_equal_rate_second_point(orc):
    # case 3 whose second point has II's own rate: I is compared with the
    # better of II's two metrics (58), and 57 < 58 keeps II.
    rt = _Retrials({(1, 0.8): (2.0, 58.0)})
    assert orc.select_fixed([2.5, 2.0], [57.0, 50.0], retrial=rt) == 1


def test_select_fixed_sequence(orc):
    """Six candidates in order, each compared with the incumbent of its turn:
    k1 dominates k0 (case 2); k2 ties k1 (case 1 keeps the incumbent); k3 is
    case 3 and stays below the incumbent's point on II's line (59.5 < 60);
    k4 is case 4 with the line at 59.6 < 60; k5 dominates (case 2)."""
    B = [3.0, 2.0, 2.0, 1.8, 2.4, 1.5]
    M = [55.0, 60.0, 60.0, 58.0, 62.0, 61.0]
    rt = _Retrials({(3, 0.8): (2.2, 61.0), (4, 1.2): (2.1, 60.2)})
    assert orc.select_fixed(B, M, retrial=rt) == 5
    assert rt.calls == [(3, 0.8), (4, 1.2)]
    # without k5 the incumbent after k1 survives
    rt = _Retrials({(3, 0.8): (2.2, 61.0), (4, 1.2): (2.1, 60.2)})
    assert orc.select_fixed(B[:5], M[:5], retrial=rt) == 1


def test_select_fixed_maxerr_mode_rate_only(orc):
    # the max-CR mode compares rates alone; equal rates keep the first
    B = [3.0, 2.0, 2.0, 2.5, 1.9, 1.9]
    M = [0.0, -1.0, 5.0, 9.0, -9.0, 9.0]
    assert orc.select_fixed(B, M, maxerr_mode=True) == 4


def test_target_mode_helpers(orc):
    # second point: above the target a larger bound, below it a smaller one
    assert orc.target_scale(61.0, 60.0) == 1.2
    assert orc.target_scale(60.0, 60.0) == 1.2
    assert orc.target_scale(59.0, 60.0) == 0.8
    # rate at the target on the line through (2.0, 58) and (2.5, 62): 2.25
    assert orc.target_rate(2.0, 58.0, 2.5, 62.0, 60.0) == pytest.approx(2.25, rel=1e-15)
    assert orc.target_rate(2.0, 61.0, 2.5, 61.0, 60.0) == 2.0
    assert math.isinf(orc.target_rate(2.0, 59.0, 2.5, 59.0, 60.0))


def test_secant_step(orc):
    # (e, M) = (1, 58) and (0.5, 66), target 60: log e moves a quarter of the
    # way from 0.5 toward 1 in log scale, e = 0.5^(1/4)
    assert orc.secant_step(1.0, 58.0, 0.5, 66.0, 60.0, 1.0, 2.0) == pytest.approx(
        0.5 ** 0.25, rel=1e-14)
    # clamped to the user bound, and to e0 / 16
    assert orc.secant_step(1.0, 58.0, 0.5, 66.0, 60.0, 1.0, 0.7) == 0.7
    assert orc.secant_step(1.0, 60.0, 0.5, 61.0, 100.0, 1.0, 2.0) == 1.0 / 16.0
    # no step: equal metrics, or a step that lands on the last bound
    assert orc.secant_step(1.0, 60.0, 0.5, 60.0, 65.0, 1.0, 2.0) is None
    assert orc.secant_step(0.5, 66.0, 1.0, 62.0, 50.0, 1.0, 1.0) is None


def test_target_pick(orc):
    e = [1.0, 1.2, 0.8, 0.9]
    M = [59.0, 58.0, 61.0, 60.5]
    # meeting 60 dB: 0.8 and 0.9 (1.2 is above the user bound 1.0) -> 0.9
    assert orc.target_pick(e, M, 60.0, 1.0) == 3
    assert orc.target_pick(e, M, 60.0, 0.85) == 2
    # nobody meets 70 dB: the smallest bound
    assert orc.target_pick(e, M, 70.0, 1.0) == 2
    # equal bounds that both meet the target: the first
    assert orc.target_pick([0.9, 0.9], [61.0, 62.0], 60.0, 1.0) == 0


@pytest.mark.parametrize("metric,eb,seed", [("PSNR", 1e-3, 11), ("SSIM", 1e-2, 21),
                                            ("AC", 1e-3, 17)])
def test_fixed_mode_replays_table1_loop(orc, metric, eb, seed):
    """orc_tune's fixed-bound mode against a replay of Sec. 6.3.2 from its
    parts: each (alpha, beta) trial in alpha-then-beta order, Table I with the
    incumbent as solution I and the new candidate as II, II's second trial at
    the bound scale Table I names.  The replay must take at least one second
    trial, so that swapping I and II or the 0.8 / 1.2 factors changes it."""
    met = getattr(orc, "METRIC_" + metric)
    x = _field(40, seed=seed)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    e = eb * vr
    o = orc.make_tune_opts(3, block=16, rate=0.08, betas=[2.0, 3.0, 4.0])
    r = orc.tune(x, e, vr, met, opts=o)
    org, bd, _ = orc.sample_blocks(x.shape, 16, 0.08)
    win = 7 if metric == "SSIM" else 0
    alphas = [1.0, 1.25, 1.5, 1.75, 2.0]
    betas = [2.0, 3.0, 4.0]

    def run(a, b, ee):
        p = orc.make_params(3, anchor_stride=16, alpha=a, beta=b)
        for ll in range(4):
            p.interp[ll], p.order[ll] = r.params.interp[ll], r.params.order[ll]
        t = orc.block_trial(x, org, bd, p, ee, ssim_win=win, ssim_step=2, vrange=vr)
        return t.B, orc.trial_metric(t, met, vr)

    cands = [(a, b) for a in alphas for b in betas]
    pts = [run(a, b, e) for a, b in cands]
    best, second = 0, 0
    for k in range(1, len(cands)):
        (bi, mi), (bk, mk) = pts[best], pts[k]
        d, sc = orc.table1(bi, mi, bk, mk)
        if d < 0:
            second += 1
            b2, m2 = run(*cands[k], sc * e)
            d, _ = orc.table1(bi, mi, bk, mk, b2, m2)
        if d == 1:
            best = k
    assert second >= 1
    assert (r.params.alpha, r.params.beta) == cands[best]
    assert r.B == pts[best][0] and r.M == pts[best][1]
    assert r.e == e
    # Algorithm 1 (4 levels x 4 candidates), the 15 candidates, the second trials
    assert r.n_trials == 16 + 15 + second


def test_select_fixed_tie_on_line_keeps_incumbent(orc):
    # II's points (2.0, 50) and (3.0, 60) put the line at exactly 55 at
    # B_I = 2.5; I at 55 lies on it, and a tie keeps the incumbent
    rt = _Retrials({(1, 0.8): (3.0, 60.0)})
    assert orc.select_fixed([2.5, 2.0], [55.0, 50.0], retrial=rt) == 0


def test_ab_candidates_alpha_outer_beta_inner(orc):
    o = orc.make_tune_opts(3, alphas=[1.0, 1.5, 2.0], betas=[2.0, 4.0])
    got = [orc.ab_candidate(o, k) for k in range(6)]
    assert got == [(1.0, 2.0), (1.0, 4.0), (1.5, 2.0), (1.5, 4.0), (2.0, 2.0), (2.0, 4.0)]
