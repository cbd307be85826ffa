"""GPU metrics against the oracle: max error exact, MSE / PSNR / SSIM within
1e-6 relative, on shapes that span several SSIM tiles with ragged edges, both
window steps of the tiled kernel, the generic path, 2-D and 3-D, and the
degenerate cases (no window fits, identical inputs, NaN)."""

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


def _pair(shape, seed, noise=0.02, offset=0.0):
    import synth
    rng = np.random.default_rng(seed)
    slope = 5.0 / 3.0 if len(shape) == 3 else 3.0
    x = (synth.grf(shape, slope=slope, seed=seed, device="cuda").cpu().numpy() + offset)
    x = x.astype(np.float32)
    y = (x + rng.uniform(-noise, noise, x.shape)).astype(np.float32)
    return x, y


def _check(q, orc, x, y, win, step, vr=None, diss_rel=1e-4):
    vr = float(x.max()) - float(x.min()) if vr is None else vr
    m = q.compute_metrics(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), vr, win, step)
    assert m.max_abs_err == orc.max_abs_err(x, y)
    assert m.mse == pytest.approx(orc.mse(x, y), rel=1e-6)
    s, nw, _ = orc.ssim(x, y, vr, win, step)
    assert m.ssim_windows == nw
    if nw == 0:
        assert math.isnan(m.ssim)
    else:
        assert m.ssim == pytest.approx(s, rel=1e-6, abs=1e-9)
        if diss_rel is not None:
            # the quantity a target SSIM compares is 1 - SSIM: match it too
            assert (1.0 - m.ssim) == pytest.approx(1.0 - s, rel=diss_rel, abs=1e-10)
    return m


@pytest.mark.parametrize("shape,step", [
    ((80, 75, 150), 2),    # 2 z-chunks, 5 y-tiles, 3 x-tiles, ragged in all three
    ((40, 23, 71), 1),     # step 1: ring of 7 planes filled every plane
    ((7, 7, 7), 2),        # exactly one window
    ((9, 30, 7), 2),
])
def test_ssim_3d_tiled(q, orc, shape, step):
    x, y = _pair(shape, seed=sum(shape))
    _check(q, orc, x, y, 7, step)


@pytest.mark.parametrize("shape,step", [((300, 700), 2), ((129, 257), 1), ((7, 64), 2)])
def test_ssim_2d_tiled(q, orc, shape, step):
    x, y = _pair(shape, seed=shape[0])
    _check(q, orc, x, y, 7, step)


@pytest.mark.parametrize("win,step", [(5, 3), (8, 4), (7, 3)])
def test_ssim_generic_windows(q, orc, win, step):
    x, y = _pair((33, 40, 45), seed=win * 10 + step)
    _check(q, orc, x, y, win, step)


def _dissimilarity_centered(x, y, vr, win, step):
    """Mean 1 - SSIM over the 3-D windows from centred moments in float64:
    each window's values are shifted by their own mean before the second
    moments are formed, so no large terms cancel (Eq. ssim, Eq. ssim2)."""
    from numpy.lib.stride_tricks import sliding_window_view as swv
    a = swv(x.astype(np.float64), (win,) * 3)[::step, ::step, ::step]
    b = swv(y.astype(np.float64), (win,) * 3)[::step, ::step, ::step]
    ax = (-3, -2, -1)
    mx, my = a.mean(axis=ax), b.mean(axis=ax)
    da, db = a - mx[..., None, None, None], b - my[..., None, None, None]
    vx, vy = (da * da).mean(axis=ax), (db * db).mean(axis=ax)
    cxy = (da * db).mean(axis=ax)
    c1, c2 = (0.01 * vr) ** 2, (0.03 * vr) ** 2
    ssim = ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2))
    return float((1.0 - ssim).mean())


def test_ssim_offset_field(q, orc):
    # Values near 1000 with errors of 1e-3: the uncentred moments of the
    # plain form cancel in 1 - SSIM (the oracle's double sums keep ~1e-3 of
    # it); SSIM itself must still agree to 1e-6, and 1 - SSIM must match a
    # centred float64 evaluation.
    x, y = _pair((40, 50, 60), seed=5, noise=1e-3, offset=1000.0)
    vr = float(x.max()) - float(x.min())
    m = _check(q, orc, x, y, 7, 2, diss_rel=None)
    assert (1.0 - m.ssim) == pytest.approx(_dissimilarity_centered(x, y, vr, 7, 2), rel=1e-4)


def test_ssim_too_small_and_identical(q, orc):
    x, y = _pair((6, 40, 40), seed=9)
    _check(q, orc, x, y, 7, 2)          # no window fits along z
    x, _ = _pair((30, 30, 30), seed=10)
    m = q.compute_metrics(torch.from_numpy(x).cuda(), torch.from_numpy(x).cuda(),
                          float(x.max() - x.min()), 7, 2)
    assert m.ssim == 1.0 and m.max_abs_err == 0.0 and math.isinf(m.psnr)


def test_metrics_nan(q, orc):
    x, y = _pair((20, 20, 20), seed=11)
    y[3, 4, 5] = np.nan
    m = q.compute_metrics(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                          float(x.max() - x.min()), 7, 2)
    assert math.isnan(m.max_abs_err) and math.isnan(orc.max_abs_err(x, y))
    assert math.isnan(m.ssim)


def test_max_err_exact_ties_and_unaligned(q, orc):
    rng = np.random.default_rng(12)
    n = 1_000_003
    x = rng.normal(0, 3, n).astype(np.float32)
    y = (x + rng.uniform(-1e-3, 1e-3, n)).astype(np.float32)
    # differences that round to the same binary32 value but differ in double
    y[100] = np.float32(x[100] + np.float32(0.01))
    y[900_000] = np.float32(x[900_000] - np.float32(0.01))
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for off in (0, 1, 3):   # 2-D views (1, n - off): unaligned starts for off > 0
        m = q.compute_metrics(xd[off:].view(1, -1), yd[off:].clone().view(1, -1), 1.0)
        assert m.max_abs_err == orc.max_abs_err(x[off:], y[off:])
        assert m.mse == pytest.approx(orc.mse(x[off:], y[off:]), rel=1e-6)


def test_ssim_256_field_vs_oracle(q, orc):
    """A field of the SSIM workload's kind (GRF plus vortex tubes) at 256^3,
    compressed at a relative bound of 1e-3 and decompressed on the GPU."""
    import synth
    x = synth.vortex_field(256, device="cuda").cpu().numpy()
    vr = float(x.max()) - float(x.min())
    xd = torch.from_numpy(x).cuda()
    blob = q.compress(xd, 1e-3)
    y = torch.empty_like(xd)
    q.decompress(blob, y)
    blob.free()
    _check(q, orc, x, y.cpu().numpy(), 7, 2, vr=vr)


# ---- Eq. (ac): autocorrelation of the compression errors

@pytest.mark.parametrize("lag", [1, 2, 7, 64])
def test_autocorr_matches_oracle(q, orc, lag):
    import synth
    a = synth.grf((40, 64, 96), 5.0 / 3.0, seed=31, n_modes=48).numpy()
    rng = np.random.default_rng(lag)
    # correlated errors of about 1e-3 (a short moving average), mean near zero
    e = np.convolve(1e-3 * rng.standard_normal(a.size), [0.6, 0.3, 0.1], mode="same")
    b = (a.ravel() + e).astype(np.float32).reshape(a.shape)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    ref = orc.autocorr(a, b, lag)
    got = q.error_autocorr(da, db, lag)
    assert got == pytest.approx(ref, abs=2e-6)
    if lag == 1:
        m = q.compute_metrics(da, db, 1.0)
        assert m.ac == pytest.approx(ref, abs=2e-6)


def test_autocorr_closed_forms(q, orc):
    n = 1 << 20
    a = torch.zeros(n, dtype=torch.float32, device="cuda")
    alt = torch.tensor([1.0, -1.0], device="cuda").repeat(n // 2)
    assert q.error_autocorr(a, alt, 1) == pytest.approx(-1.0, abs=1e-12)
    assert q.error_autocorr(a, alt, 2) == pytest.approx(1.0, abs=1e-12)
    # constant error: no variance, AC 0 (as the oracle's exact zero)
    assert q.error_autocorr(a, torch.full_like(a, 0.25), 1) == 0.0
    # lag at or past the end
    assert q.error_autocorr(a[:5], alt[:5], 5) == 0.0
    # ragged length, unaligned start
    x = torch.randn(100003, device="cuda")
    y = x + 1e-3 * torch.randn(100003, device="cuda")
    ref = orc.autocorr(x[1:].cpu().numpy(), y[1:].cpu().numpy(), 3)
    assert q.error_autocorr(x[1:], y[1:], 3) == pytest.approx(ref, abs=2e-6)
