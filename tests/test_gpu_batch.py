"""Batched compression (one launch per level and kernel instance across
fields, replayed as a CUDA graph, tile variants timed): every field's blob
must be bit-identical to the oracle's compression of that field, and to the
single-field path, on mixed 2-D / 3-D batches with ragged shapes, mixed
parameters, relative and absolute bounds, repeated runs with new data,
long unpredictable lists (device sort limit and list overflow)."""

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


def _blob_arrays(blob):
    codes, ui, uv, an = blob.arrays()
    hist = blob.histogram()
    torch.cuda.synchronize()
    return (codes.cpu().numpy().view(np.uint16), ui.cpu().numpy(),
            uv.cpu().numpy().view(np.uint32), an.cpu().numpy().view(np.uint32),
            hist.numpy().astype(np.uint64), blob.info())


def _same_blob(a, b):
    ca, ia, va, aa, ha, fa = _blob_arrays(a)
    cb, ib, vb, ab, hb, fb = _blob_arrays(b)
    assert np.array_equal(ca, cb), "codes"
    assert np.array_equal(ia, ib) and np.array_equal(va, vb), "unpredictable list"
    assert np.array_equal(aa, ab), "anchors"
    assert np.array_equal(ha, hb), "histogram"
    assert fa.abs_eb == fb.abs_eb and fa.n_unpredictable == fb.n_unpredictable
    assert fa.est_bits == fb.est_bits


def _vs_oracle(orc, blob, x, e, op):
    c, ui, uv, an, h, info = _blob_arrays(blob)
    ref = orc.compress(x, e, op)
    assert info.abs_eb == e
    assert np.array_equal(c, ref["codes"]), "codes"
    assert np.array_equal(ui, ref["unpred_idx"]), "unpredictable indices"
    assert np.array_equal(uv, ref["unpred_val"].view(np.uint32)), "unpredictable values"
    assert np.array_equal(an, ref["anchors"].view(np.uint32)), "anchors"
    assert np.array_equal(h, orc.histogram(ref["codes"], op.anchor_stride)), "histogram"


def _fields(seed, shapes):
    import synth
    rng = np.random.default_rng(seed)
    out = []
    for i, s in enumerate(shapes):
        slope = 5.0 / 3.0 if len(s) == 3 else 3.0
        x = synth.grf(s, slope, seed=seed * 100 + i, n_modes=64, device="cuda")
        x = x + torch.from_numpy(rng.normal(0, 0.02, s).astype(np.float32)).cuda()
        out.append(x.contiguous())
    return out


SHAPES = [(37, 50, 150), (300, 517), (33, 33, 33), (64, 128), (20, 70, 41), (9, 9, 200),
          (129, 65)]


def _params(q, orc, shapes, seed):
    rng = np.random.default_rng(seed)
    qps, ops = [], []
    for s in shapes:
        nd = len(s)
        nl = 5 if nd == 3 else 6
        interp = [int(v) for v in rng.integers(0, 2, nl)]
        order = [int(v) for v in rng.integers(0, 6 if nd == 3 else 2, nl)]
        alpha = float(rng.choice([1.0, 1.25, 1.5, 2.0]))
        beta = float(rng.choice([1.5, 2.0, 4.0]))
        qps.append(q.make_params(nd, interp=interp, order=order, alpha=alpha, beta=beta))
        ops.append(orc.make_params(nd, interp=interp, order=order, alpha=alpha, beta=beta))
    return qps, ops


@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_oracle_and_single(q, orc, graph):
    fields = _fields(1, SHAPES)
    qps, ops = _params(q, orc, SHAPES, 7)
    plan = q.Batch(SHAPES, qps, graph=graph)
    for run in range(2):   # second run: new data through the same plan / graph
        if run == 1:
            fields = _fields(2, SHAPES)
        blobs = plan.compress(fields, 1e-3)
        for x, b, qp, op in zip(fields, blobs, qps, ops):
            xn = x.cpu().numpy()
            mn, mx, _ = orc.value_range(xn)
            _vs_oracle(orc, b, xn, 1e-3 * (float(mx) - float(mn)), op)
            single = q.compress(x, 1e-3, qp)
            _same_blob(b, single)
            single.free()
            b.free()
    inf = plan.info()
    assert inf.graph == (1 if graph else 0)
    assert inf.nfields == len(SHAPES) and inf.n_groups > 0
    plan.free()


def test_batch_absolute_bounds_and_autotune(q, orc):
    fields = _fields(3, SHAPES)
    qps, ops = _params(q, orc, SHAPES, 8)
    ebs = [0.01, 0.002, 0.05, 0.0, 0.03, 0.004, 0.02]
    plan = q.Batch(SHAPES, qps, autotune=True)
    blobs = plan.compress(fields, ebs, relative=False)
    inf = plan.info()
    assert inf.autotuned == 1 and inf.level1_groups >= 1
    for i in range(min(16, inf.level1_groups)):
        assert inf.level1_variant[i] in (0, 1, 2, 3)
        assert inf.level1_ms[i][0] > 0 and inf.level1_ms[i][1] > 0
    for x, b, e, op in zip(fields, blobs, ebs, ops):
        _vs_oracle(orc, b, x.cpu().numpy(), e, op)
        b.free()
    plan.free()


# every row starts on a 16-byte boundary: level 1 takes the bulk tensor copies
BULK_SHAPES = [(37, 50, 148), (64, 128), (33, 33, 36), (300, 520), (20, 70, 40)]


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_bulk_copies_match_oracle(q, orc, autotune):
    fields = _fields(7, BULK_SHAPES)
    qps, ops = _params(q, orc, BULK_SHAPES, 10)
    plan = q.Batch(BULK_SHAPES, qps, autotune=autotune)
    for run in range(2):
        if run == 1:
            fields = _fields(8, BULK_SHAPES)
        blobs = plan.compress(fields, 1e-3)
        for x, b, qp, op in zip(fields, blobs, qps, ops):
            xn = x.cpu().numpy()
            mn, mx, _ = orc.value_range(xn)
            _vs_oracle(orc, b, xn, 1e-3 * (float(mx) - float(mn)), op)
            b.free()
    inf = plan.info()
    if not autotune:
        # 3-D groups: the persistent kernel (3); 2-D groups: one tile per CTA (2)
        assert all(inf.level1_variant[i] in (2, 3) for i in range(inf.level1_groups))
        assert any(inf.level1_variant[i] == 3 for i in range(inf.level1_groups))
    plan.free()


def test_batch_long_lists(q, orc):
    """One field with ~5000 unpredictable points (longer than the on-device
    sort), one whose list overflows the plan's capacity (the field is redone
    through the single-field path), and one ordinary field."""
    rng = np.random.default_rng(5)
    shapes = [(40, 40, 40), (300, 300), (17, 19, 23)]
    fields = _fields(4, shapes)
    a = fields[0].cpu().numpy()
    idx = rng.choice(a.size, 5000, replace=False)
    a.reshape(-1)[idx] = rng.uniform(1e4, 1e5, idx.size).astype(np.float32)
    fields[0] = torch.from_numpy(a).cuda()
    fields[1] = torch.from_numpy(rng.uniform(-1, 1, shapes[1]).astype(np.float32)).cuda()
    qps, ops = _params(q, orc, shapes, 9)
    plan = q.Batch(shapes, qps)
    ebs = [1e-3, 1e-9, 1e-3]
    blobs = plan.compress(fields, ebs, relative=False)
    assert blobs[0].info().n_unpredictable > 2048
    assert blobs[1].info().n_unpredictable > 65536
    for x, b, e, op in zip(fields, blobs, ebs, ops):
        _vs_oracle(orc, b, x.cpu().numpy(), e, op)
        b.free()
    plan.free()


def test_compress_batch_one_shot_and_decompress(q, orc):
    fields = _fields(6, SHAPES[:4])
    blobs = q.compress_batch(fields, 1e-4)
    for x, b in zip(fields, blobs):
        single = q.compress(x, 1e-4)
        _same_blob(b, single)
        y = q.decompress(b)
        ys = q.decompress(single)
        assert torch.equal(y.view(torch.int32), ys.view(torch.int32))
        single.free()
        b.free()


def test_batch_rejects_bad_input(q):
    plan = q.Batch([(10, 10, 10)])
    x = torch.zeros((10, 10, 10), device="cuda")
    with pytest.raises(q.QozError):
        plan.compress([x], -1.0)
    with pytest.raises(q.QozError):
        q.Batch([(10, 10, 10, 10)])
    plan.free()


def test_batch_bulk_copy_wait_times_out_cleanly(q, orc, monkeypatch):
    """A bulk-copy tile whose barrier never completes fails the whole batch
    with QOZ_ETIMEOUT (host fault injection: the barrier's second phase
    expects bytes no copy brings; the copies themselves have landed), and
    the next run of the same plan, graph and all, is exact again."""
    fields = _fields(11, BULK_SHAPES)
    qps, ops = _params(q, orc, BULK_SHAPES, 12)
    plan = q.Batch(BULK_SHAPES, qps)
    monkeypatch.setenv("QOZ_FAULT", "tma_wait")
    with pytest.raises(q.QozError) as ei:
        plan.compress(fields, 1e-3)
    assert ei.value.status == 5
    monkeypatch.delenv("QOZ_FAULT")
    blobs = plan.compress(fields, 1e-3)
    for x, b, op in zip(fields, blobs, ops):
        xn = x.cpu().numpy()
        mn, mx, _ = orc.value_range(xn)
        _vs_oracle(orc, b, xn, 1e-3 * (float(mx) - float(mn)), op)
        b.free()
    plan.free()
