"""Concurrent use of the library: host threads, each on its own CUDA stream,
tune, compress, decompress and serialize different fields at the same time,
repeatedly; every result must be bit-identical to the same call made alone.
(The library's host state is per thread or guarded; device scratch comes
from the stream-ordered pool, whose reuse across streams waits for the free
to complete.)"""

import threading

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


def _run(q, x, opts, stream):
    with torch.cuda.stream(stream):
        rep = q.tune(x, 1e-3, q.METRIC_PSNR, float("nan"), opts, stream=stream)
        blob = q.compress_abs(x, rep.abs_eb, rep.params, stream=stream)
        y = q.decompress(blob, stream=stream)
        ser = blob.serialize(stream=stream)
        codes = blob.arrays(stream=stream)[0]
        stream.synchronize()
        out = (rep.abs_eb, list(rep.params.interp), list(rep.params.order), rep.params.alpha,
               rep.params.beta, rep.B, rep.M, codes.cpu().numpy().copy(),
               y.cpu().numpy().view(np.uint32).copy(), ser.numpy().copy())
        blob.free()
    return out


def test_threads_on_streams_match_serial(q):
    import synth
    shapes = [(64, 64, 64), (48, 70, 90), (1, 300, 517), (37, 50, 148)]
    fields = [synth.grf(s, 5.0 / 3.0, seed=40 + i, n_modes=32).cuda().contiguous()
              for i, s in enumerate(shapes)]
    opts = q.make_tune_opts(block=16, rate=0.1, n_orders=6)
    s0 = torch.cuda.current_stream()
    ref = [_run(q, f, opts, s0) for f in fields]
    results = [[] for _ in fields]
    errors = []

    def worker(i):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            for _ in range(3):
                results[i].append(_run(q, fields[i], opts, st))
        except Exception as ex:  # reported below
            errors.append(repr(ex))

    ths = [threading.Thread(target=worker, args=(i,)) for i in range(len(fields))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errors, errors
    for i, r in enumerate(ref):
        assert len(results[i]) == 3
        for got in results[i]:
            assert got[:7] == r[:7], f"field {i}: tuner report differs"
            for k in (7, 8, 9):
                assert np.array_equal(got[k], r[k]), f"field {i}: array {k} differs"
