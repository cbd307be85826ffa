"""The ablation of Sec. 7.2.4 on a small synthetic field: the five settings
(SZ3-like, +AP, +S, +LIS, QoZ) are derived as the benchmark's ablation
workload derives them, the choices of the sampled steps equal the oracle's,
and each setting's compression is bit-exact against the oracle."""

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


def test_ablation_variants(q, orc):
    from test_gpu_parity import run_parity
    import synth
    n = 64
    x = (synth.grf((n, n, n), 5.0 / 3.0, seed=2, n_modes=96)
         + synth.fronts((n, n, n), 2000, count=3)).numpy()
    xd = torch.from_numpy(x).cuda()
    rel = 1e-3
    alphas, betas = [1.0, 1.5, 2.0], [2.0, 4.0]
    opts = q.make_tune_opts(block=16, rate=0.05, n_orders=6, alphas=alphas, betas=betas)
    oopts = orc.make_tune_opts(3, block=16, rate=0.05, n_orders=6, alphas=alphas, betas=betas)
    mn, mx, _ = orc.value_range(x)
    vr = float(mx) - float(mn)
    e = rel * vr
    # +S: the single (interpolator, order) with the lowest sampled bit rate
    org, bd, _ = orc.sample_blocks(x.shape, 16, 0.05)
    assert org.shape[0] > 1
    best = None
    for interp in (0, 1):
        for od in range(6):
            v = q.tune_verify(xd, rel, q.make_params(3, interp=interp, order=od), opts=opts)
            t = orc.block_trial(x, org, bd, orc.make_params(3, interp=interp, order=od,
                                                              anchor_stride=16), e, vrange=vr)
            assert v.B == pytest.approx(t.B, rel=1e-12)
            if best is None or v.B < best[0]:
                best = (v.B, interp, od)
    # +LIS and QoZ: the tuner's level-wise choices and its (alpha, beta)
    rep = q.tune(xd, rel, q.METRIC_MAXERR, float("nan"), opts)
    ref = orc.tune(x, e, vr, orc.METRIC_MAXERR, opts=oopts)
    assert list(rep.params.interp[:5]) == list(ref.params.interp[:5])
    assert list(rep.params.order[:5]) == list(ref.params.order[:5])
    assert (rep.params.alpha, rep.params.beta) == (ref.params.alpha, ref.params.beta)
    lis_i, lis_o = list(rep.params.interp[:5]), list(rep.params.order[:5])
    variants = {
        "sz3": dict(interp=1, order=0, alpha=1.0, beta=1.0, stride=256),
        "ap": dict(interp=1, order=0, alpha=1.0, beta=1.0, stride=32),
        "ap_s": dict(interp=best[1], order=best[2], alpha=1.0, beta=1.0, stride=32),
        "ap_s_lis": dict(interp=lis_i, order=lis_o, alpha=1.0, beta=1.0, stride=32),
        "qoz": dict(interp=lis_i, order=lis_o, alpha=rep.params.alpha, beta=rep.params.beta,
                    stride=32),
    }
    for name, v in variants.items():
        refc, ee = run_parity(q, orc, x, rel, **v)
        assert ee == e
        err = np.abs(x.astype(np.float64) - refc["recon"].astype(np.float64))
        assert err.max() <= e, name
