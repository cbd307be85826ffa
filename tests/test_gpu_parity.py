"""GPU parity: the CUDA path (through the C ABI) against the oracle, element
by element on the same seeded inputs.  Codes, unpredictable lists, anchors
and reconstructions must be bit-exact; the Huffman rate estimate is exact
(integer histograms); metrics agree within 1e-6 relative."""

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


def _params(q, orc, nd, interp, order, alpha, beta, stride=0):
    qp = q.make_params(nd, interp=interp, order=order, alpha=alpha, beta=beta,
                       anchor_stride=stride)
    op = orc.make_params(nd, interp=interp, order=order, alpha=alpha, beta=beta,
                         anchor_stride=stride or None)
    return qp, op


def run_parity(q, orc, x, rel=1e-3, interp=1, order=0, alpha=1.5, beta=4.0, stride=0,
               abs_eb=None):
    x = np.ascontiguousarray(x, dtype=np.float32)
    nd = x.ndim
    qp, op = _params(q, orc, nd, interp, order, alpha, beta, stride)
    xd = torch.from_numpy(x).cuda()
    recon = torch.empty_like(xd)
    if abs_eb is None:
        blob = q.compress(xd, rel, qp, recon=recon)
        mn, mx, _ = orc.value_range(x)
        e = rel * (float(mx) - float(mn))
    else:
        blob = q.compress_abs(xd, abs_eb, qp, recon=recon)
        e = abs_eb
    out = q.decompress(blob)
    codes, ui, uv, an = blob.arrays()
    hist = blob.histogram()
    torch.cuda.synchronize()
    info = blob.info()
    ref = orc.compress(x, e, op)
    assert info.abs_eb == e
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), ref["codes"]), "codes"
    assert np.array_equal(an.cpu().numpy().view(np.uint32), ref["anchors"].view(np.uint32))
    assert np.array_equal(ui.cpu().numpy(), ref["unpred_idx"]), "unpredictable indices"
    assert np.array_equal(uv.cpu().numpy().view(np.uint32), ref["unpred_val"].view(np.uint32))
    rb = ref["recon"].view(np.uint32)
    assert np.array_equal(recon.cpu().numpy().view(np.uint32), rb), "compress-side recon"
    assert np.array_equal(out.cpu().numpy().view(np.uint32), rb), "decompressed field"
    oh = orc.histogram(ref["codes"], op.anchor_stride)
    assert np.array_equal(hist.numpy().astype(np.uint64), oh), "histogram"
    assert info.est_bits == orc.estimate_bits(oh, len(ref["unpred_idx"]), len(ref["anchors"]))
    blob.free()
    return ref, e


def test_trend_field_plain_method(q, orc):
    """64^3 k^-5/3 field + trend, eps 1e-3, cubic, order z,y,x, alpha 1.5,
    beta 4: the plain-method configuration."""
    import synth
    x = synth.grf_trend_field(64).numpy()
    ref, e = run_parity(q, orc, x, 1e-3, interp=1, order=0, alpha=1.5, beta=4.0)
    err = np.abs(x.astype(np.float64) - ref["recon"].astype(np.float64))
    assert err.max() <= e


@pytest.mark.parametrize("order", range(6))
@pytest.mark.parametrize("interp", [0, 1])
def test_orders_uneven_3d(q, orc, order, interp):
    # spans several tiles along every axis with ragged tails
    rng = np.random.default_rng(100 + order)
    import synth
    x = synth.grf((37, 50, 150), 5.0 / 3.0, seed=10 + order, n_modes=96).numpy()
    x += rng.normal(0, 0.05, x.shape).astype(np.float32)
    run_parity(q, orc, x, 1e-3, interp=interp, order=order, alpha=1.25, beta=3.0)


@pytest.mark.parametrize("order", range(6))
@pytest.mark.parametrize("shape", [(37, 50, 148), (45, 70, 136)])
def test_orders_bulk_copy_shapes(q, orc, order, shape):
    # rows of 148 / 136 values start on 16-byte boundaries: level 1 takes the
    # bulk tensor copies (loads only for 148, loads and the code store for
    # 136), with ragged tiles on every axis
    import synth
    x = synth.grf(shape, 5.0 / 3.0, seed=20 + order, n_modes=96).numpy()
    run_parity(q, orc, x, 1e-3, interp=order % 2, order=order, alpha=1.5, beta=2.0)


@pytest.mark.parametrize("order", range(6))
@pytest.mark.parametrize("shape", [(40, 72, 200), (100, 44, 96)])
def test_level1_persistent_orders(q, orc, order, shape):
    # rows of 200 / 96 values keep every array's rows on 16-byte boundaries,
    # so level 1 runs on the persistent bulk-copy kernel: tiles on every edge
    # and inside, ragged tails on z, y and x, both interpolators
    import synth
    x = synth.grf(shape, 5.0 / 3.0, seed=40 + order, n_modes=96).numpy()
    for interp in (0, 1):
        run_parity(q, orc, x, 1e-3, interp=interp, order=order, alpha=1.25, beta=3.0)


def test_level1_many_tiles_per_cta(q, orc):
    # 256^3: thousands of tiles over the resident CTAs, so each CTA reuses
    # both pipeline stages and both code buffers many times
    import synth
    x = synth.grf((256, 256, 256), 5.0 / 3.0, seed=77, n_modes=128).numpy()
    for order in (3, 4):
        run_parity(q, orc, x, 1e-4, interp=1, order=order, alpha=1.5, beta=2.0)


def test_mixed_levels(q, orc):
    import synth
    x = synth.grf((70, 45, 99), 2.5, seed=3, n_modes=64).numpy()
    run_parity(q, orc, x, 1e-4, interp=[0, 1, 0, 1, 1], order=[5, 2, 4, 1, 3], alpha=2.0,
               beta=1.5)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("interp", [0, 1])
def test_2d(q, orc, order, interp):
    import synth
    x = (synth.zonal_bands(300, 517, 3001) + synth.grf((300, 517), 3.0, seed=3001,
                                                          sigma=1.0)).numpy()
    run_parity(q, orc, x, 1e-3, interp=interp, order=order, alpha=1.75, beta=2.0)


def test_2d_cesm_shape(q, orc):
    import synth
    x = (synth.zonal_bands(1800, 3600, 3000) + synth.grf((1800, 3600), 3.0, seed=3000,
                                                            sigma=1.0)).numpy()
    run_parity(q, orc, x, 1e-3, interp=1, order=1, alpha=1.5, beta=3.0)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 5), (1, 40, 33), (7, 1, 9), (33, 33, 33),
                                   (65, 2, 64), (1, 1), (1, 100), (100, 1), (3, 2)])
def test_degenerate_shapes(q, orc, shape):
    rng = np.random.default_rng(7)
    x = np.cumsum(rng.standard_normal(shape), axis=-1).astype(np.float32)
    nd = len(shape)
    for order in range(6 if nd == 3 else 2):
        run_parity(q, orc, x, 1e-2, interp=1, order=order, alpha=1.5, beta=2.0)


@pytest.mark.parametrize("stride", [2, 4, 8, 16, 64, 128, 256])
def test_anchor_strides(q, orc, stride):
    import synth
    x = synth.grf((40, 41, 90), 5.0 / 3.0, seed=5, n_modes=64).numpy()
    run_parity(q, orc, x, 1e-3, interp=1, order=2, alpha=1.5, beta=4.0, stride=stride)


def test_nonfinite_values(q, orc):
    rng = np.random.default_rng(11)
    x = np.cumsum(rng.standard_normal((30, 40, 50)), axis=2).astype(np.float32)
    x[3, 4, 5] = np.nan
    x[10, 0, 0] = np.inf
    x[0, 0, 0] = -np.inf          # an anchor
    x[29, 39, 49] = np.nan
    run_parity(q, orc, x, 1e-3)


def test_constant_field_zero_bound(q, orc):
    x = np.full((20, 30, 40), -2.5, np.float32)
    ref, e = run_parity(q, orc, x, 1e-3)
    assert e == 0.0 and len(ref["unpred_idx"]) == 0


def test_absolute_bound(q, orc):
    import synth
    x = synth.grf((48, 48, 48), 2.0, seed=21, n_modes=64).numpy()
    run_parity(q, orc, x, abs_eb=0.01, interp=0, order=3, alpha=1.0, beta=1.0)


@pytest.mark.parametrize("n_extra", [50, 5000])
def test_many_unpredictables(q, orc, n_extra):
    # large magnitudes with a tiny absolute bound make reconstruction rounding
    # miss the bound: exercises the unpredictable list and its ordering (the
    # in-block and the multi-launch sort paths)
    rng = np.random.default_rng(13)
    x = rng.normal(0, 1, (40, 60, 80)).astype(np.float32)
    idx = rng.choice(x.size, size=n_extra, replace=False)
    x.reshape(-1)[idx] = rng.uniform(1e6, 1e7, n_extra).astype(np.float32)
    ref, _ = run_parity(q, orc, x, abs_eb=1e-3, interp=1, order=0, alpha=1.0, beta=1.0)
    assert len(ref["unpred_idx"]) > (10 if n_extra == 50 else 2048)


def test_value_range(q, orc):
    rng = np.random.default_rng(17)
    x = rng.normal(0, 3, 1_000_003).astype(np.float32)
    x[5] = np.nan
    x[77] = np.inf
    xd = torch.from_numpy(x).cuda()
    for off in (0, 1, 2, 3):          # unaligned starts take the scalar head
        mn, mx, cnt = q.value_range(xd[off:])
        omn, omx, ocnt = orc.value_range(x[off:])
        assert (mn, mx, cnt) == (omn, omx, ocnt)


def test_metrics(q, orc):
    import synth
    x = synth.grf_trend_field(48).numpy()
    y = (x + np.random.default_rng(3).normal(0, 0.02, x.shape)).astype(np.float32)
    vr = float(x.max()) - float(x.min())
    m = q.compute_metrics(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), vr, 7, 2)
    assert m.max_abs_err == orc.max_abs_err(x, y)
    assert m.mse == pytest.approx(orc.mse(x, y), rel=1e-6)
    assert m.psnr == pytest.approx(orc.psnr(x, y, vr), rel=1e-6)
    s, nw, _ = orc.ssim(x, y, vr, 7, 2)
    assert m.ssim_windows == nw
    assert m.ssim == pytest.approx(s, rel=1e-6)
    x2 = x[0]
    y2 = y[0]
    m2 = q.compute_metrics(torch.from_numpy(x2.copy()).cuda(), torch.from_numpy(y2.copy()).cuda(),
                           vr, 7, 1)
    s2, nw2, _ = orc.ssim(x2, y2, vr, 7, 1)
    assert m2.ssim_windows == nw2 and m2.ssim == pytest.approx(s2, rel=1e-6)
    same = q.compute_metrics(torch.from_numpy(x).cuda(), torch.from_numpy(x).cuda(), vr)
    assert same.max_abs_err == 0.0 and math.isinf(same.psnr)


def test_serialize_round_trip_and_corruption(q, orc):
    import synth
    x = synth.grf((40, 50, 60), 5.0 / 3.0, seed=8, n_modes=64).numpy()
    x[1, 2, 3] = np.nan
    xd = torch.from_numpy(x).cuda()
    recon = torch.empty_like(xd)
    blob = q.compress(xd, 1e-3, q.make_params(3, alpha=1.5, beta=4), recon=recon)
    buf = blob.serialize()
    b2 = q.deserialize(buf.clone())
    out = q.decompress(b2)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), recon.cpu().numpy().view(np.uint32))
    assert np.array_equal(b2.histogram().numpy(), blob.histogram().numpy())
    bad = buf.clone()
    bad[len(bad) // 2] ^= 0x10
    with pytest.raises(q.QozError) as ei:
        q.deserialize(bad)
    assert ei.value.status == 4
    with pytest.raises(q.QozError):
        q.deserialize(buf[: len(buf) - 9].clone())


def test_serialize_async_matches_sync(q):
    import synth
    x = synth.grf((33, 47, 64), 5.0 / 3.0, seed=9, n_modes=64).cuda()
    blob = q.compress(x, 1e-3)
    ref = blob.serialize()
    s = torch.cuda.Stream()
    out = torch.full((ref.numel() + 64,), 0xAB, dtype=torch.uint8, pin_memory=True)
    used = blob.serialize_async(out, stream=s)
    s.synchronize()
    assert used == ref.numel()
    assert torch.equal(out[:used], ref)
    b2 = q.deserialize(out[:used].clone())
    assert b2.info().n_unpredictable == blob.info().n_unpredictable
    blob.free()
    b2.free()


def test_profile_stage_mask(q):
    # only the selected stages record events; the launch counter always runs
    import synth
    x = synth.grf((40, 48, 64), 5.0 / 3.0, seed=4, n_modes=32).cuda()
    q.profile_read(reset=True)
    q.profile_enable(True, stages=[q.STAGE_LEVEL + 1])
    q.compress(x, 1e-3).free()
    torch.cuda.synchronize()
    q.profile_enable(False)
    t = q.profile_read(reset=True)
    assert t.calls[q.STAGE_LEVEL + 1] == 1 and t.ms[q.STAGE_LEVEL + 1] > 0
    assert sum(t.calls[i] for i in range(32) if i != q.STAGE_LEVEL + 1) == 0
    assert t.launches > 0
    q.profile_enable(True)  # all stages again
    q.compress(x, 1e-3).free()
    torch.cuda.synchronize()
    q.profile_enable(False)
    t = q.profile_read(reset=True)
    assert t.calls[q.STAGE_RANGE] == 1 and t.calls[q.STAGE_LEVEL + 2] == 1


def test_bulk_copy_wait_times_out_cleanly(q, monkeypatch):
    # the level-1 tile barrier is told to expect 16 bytes more than its
    # copies bring: every tile's bounded wait runs out, the launch reports
    # the timeout, and the context stays usable
    x = torch.rand((40, 48, 64), device="cuda")
    monkeypatch.setenv("QOZ_FAULT", "tma_wait")
    with pytest.raises(q.QozError) as ei:
        q.compress(x, 1e-3)
    assert ei.value.status == 5
    monkeypatch.delenv("QOZ_FAULT")
    b = q.compress(x, 1e-3)
    assert b.info().n_points == x.numel()
    b.free()


def test_host_fault_injection(q, monkeypatch):
    x = torch.zeros((16, 16, 16), device="cuda")
    monkeypatch.setenv("QOZ_FAULT", "alloc")
    with pytest.raises(q.QozError) as ei:
        q.compress(x, 1e-3)
    assert ei.value.status == 2
    monkeypatch.setenv("QOZ_FAULT", "launch")
    with pytest.raises(q.QozError) as ei:
        q.compress(x, 1e-3)
    assert ei.value.status == 3
    monkeypatch.delenv("QOZ_FAULT")
    blob = q.compress(x, 1e-3)            # the context is still usable
    buf = blob.serialize()
    monkeypatch.setenv("QOZ_FAULT", "header")
    with pytest.raises(q.QozError) as ei:
        q.deserialize(buf.clone())
    assert ei.value.status == 4


def test_invalid_arguments(q):
    x = torch.zeros((8, 8, 8), device="cuda")
    for bad in (0.0, -1e-3, float("nan"), float("inf")):
        with pytest.raises(q.QozError):
            q.compress(x, bad)
    with pytest.raises(q.QozError):
        q.compress(x, 1e-3, q.make_params(3, alpha=0.5))
    with pytest.raises(q.QozError):
        q.compress(x, 1e-3, q.make_params(3, order=6))
    with pytest.raises(q.QozError):
        q.compress(x, 1e-3, q.make_params(3, anchor_stride=24))
    with pytest.raises(q.QozError):
        q.compress(torch.zeros((4, 4, 4, 4), device="cuda"), 1e-3)


@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-4])
def test_full_size_512(q, orc, eps):
    """512^3 (NYX-sized) field with fronts at the three bounds of the
    plain-method-at-scale case, whole-field parity in the launch
    configuration the benchmark times."""
    import synth
    xg = synth.grf_fronts_field(512, device="cuda")
    x = xg.cpu().numpy()
    del xg
    run_parity(q, orc, x, eps, interp=1, order=0, alpha=1.5, beta=4.0)


def test_binding_rejects_wrong_sized_buffers(q):
    # the checks raise in the binding before the library is called
    x = torch.randn((8, 9, 10), device="cuda")
    with pytest.raises(ValueError):
        q.compress(x, 1e-3, recon=torch.empty(719, device="cuda"))
    with pytest.raises(ValueError):
        q.compress_abs(x, 1e-2, recon=torch.empty(721, device="cuda"))
    blob = q.compress(x, 1e-3)
    with pytest.raises(ValueError):
        q.decompress(blob, torch.empty(10, device="cuda"))
    with pytest.raises(ValueError):
        blob.serialize(out=torch.empty(1 << 16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ValueError):
        blob.serialize_async(torch.empty(1 << 16, dtype=torch.uint8, device="cuda"))
    y = q.decompress(blob, torch.empty(720, device="cuda"))  # any shape of the same size
    assert y.numel() == 720
    blob.free()


def test_decompress_flags_missing_unpredictable_entry(q):
    """A code-0 point whose index is missing from the unpredictable list (a
    corrupt blob that no checksum caught) decompresses to 0.0 and is
    reported by qoz_blob_check as QOZ_ECORRUPT; an intact blob checks OK."""
    import ctypes as C
    x = torch.randn((16, 24, 40), device="cuda").cumsum(2)
    x[3, 4, 5] = float("nan")
    x[9, 1, 33] = float("inf")
    blob = q.compress(x, 1e-3)
    y = q.decompress(blob)
    blob.check()
    pidx = C.c_void_p()
    n = C.c_int64()
    q.lib().qoz_blob_arrays(blob.handle, None, C.byref(pidx), None, C.byref(n), None, None)
    assert n.value >= 2

    class _Dev:
        __cuda_array_interface__ = {"shape": (n.value,), "typestr": "<i8",
                                    "data": (pidx.value, False), "version": 3}

    idx = torch.as_tensor(_Dev(), device="cuda")
    lost = int(idx[0].item())
    idx[0] = -1                      # still sorted; the first listed point loses its entry
    y = q.decompress(blob)
    with pytest.raises(q.QozError) as ei:
        blob.check()
    assert ei.value.status == 4
    assert y.view(-1)[lost].item() == 0.0
    idx[0] = lost                    # restored: decompression is clean again
    q.decompress(blob, out=y)
    blob.check()
    blob.free()


def test_full_size_1024_benchmark_configuration(q, orc):
    """The 1024^3 headline field (4 GiB) in the launch configuration the
    benchmark times: the sampled tuner's setting (max-CR mode, 0.5 % of the
    field in 33^3 blocks, 12 interpolators, alpha x beta), then the
    compression at the tuner's absolute bound; codes, lists, anchors and
    both reconstructions bit-exact against the oracle with the same setting
    and bound."""
    import synth
    xg = synth.grf_fronts_field(1024, device="cuda")
    topts = q.make_tune_opts(block=32, rate=0.005, n_orders=6,
                             alphas=[1.0, 1.25, 1.5, 1.75, 2.0], betas=[2.0, 3.0, 4.0])
    rep = q.tune(xg, 1e-3, q.METRIC_MAXERR, float("nan"), topts)
    x = xg.cpu().numpy()
    mn, mx, _ = orc.value_range(x)
    assert rep.abs_eb == 1e-3 * (float(mx) - float(mn))
    interp = [int(v) for v in rep.params.interp[:5]]
    order = [int(v) for v in rep.params.order[:5]]
    recon = torch.empty_like(xg)
    blob = q.compress_abs(xg, rep.abs_eb, rep.params, recon=recon)
    codes, ui, uv, an = blob.arrays()
    hist = blob.histogram()
    torch.cuda.synchronize()
    op = orc.make_params(3, interp=interp, order=order, alpha=rep.params.alpha,
                         beta=rep.params.beta)
    ref = orc.compress(x, rep.abs_eb, op)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), ref["codes"]), "codes"
    del codes
    assert np.array_equal(an.cpu().numpy().view(np.uint32), ref["anchors"].view(np.uint32))
    assert np.array_equal(ui.cpu().numpy(), ref["unpred_idx"])
    assert np.array_equal(uv.cpu().numpy().view(np.uint32), ref["unpred_val"].view(np.uint32))
    rb = ref["recon"].view(np.uint32)
    assert np.array_equal(recon.cpu().numpy().view(np.uint32), rb), "compress-side recon"
    del recon
    out = q.decompress(blob)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), rb), "decompressed field"
    blob.check()
    oh = orc.histogram(ref["codes"], op.anchor_stride)
    assert np.array_equal(hist.numpy().astype(np.uint64), oh), "histogram"
    blob.free()
