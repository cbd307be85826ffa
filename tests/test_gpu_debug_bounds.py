"""The bounds-checking build (QOZ_DEBUG_BOUNDS): every checked shared- and
global-memory index of the level, trial and entropy kernels is compared with
its array's extent, and a failure is recorded and skipped rather than
trapping (compute-sanitizer is not available).  A child process loads that
build, runs compression, decompression, the tuners, metrics, serialization
and a batch on awkward shapes, checks the results against the oracle, and
requires an empty record."""

import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
import oracle as orc
import paper_2310_14133_gb300 as q
import synth

orc.build()
q.debug_bounds(reset=True)
out = {"cases": 0}

def parity(x, rel, interp, order, alpha, beta, stride=0):
    x = np.ascontiguousarray(x, dtype=np.float32)
    nd = x.ndim
    qp = q.make_params(nd, interp=interp, order=order, alpha=alpha, beta=beta,
                       anchor_stride=stride)
    op = orc.make_params(nd, interp=interp, order=order, alpha=alpha, beta=beta,
                         anchor_stride=stride or None)
    xd = torch.from_numpy(x).cuda()
    blob = q.compress(xd, rel, qp)
    mn, mx, _ = orc.value_range(x)
    ref = orc.compress(x, rel * (float(mx) - float(mn)), op)
    codes = blob.arrays()[0].cpu().numpy().view(np.uint16)
    assert np.array_equal(codes, ref["codes"]), "codes"
    y = q.decompress(blob)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), ref["recon"].view(np.uint32)), "recon"
    b2 = q.deserialize(blob.serialize())
    assert torch.equal(b2.arrays()[0], blob.arrays()[0]), "serialized codes"
    b2.free()
    blob.free()
    out["cases"] += 1

for shape in [(1, 1, 1), (2, 3, 5), (7, 1, 9), (33, 33, 33), (1, 40, 33), (17, 65, 130)]:
    x = synth.grf(shape, 5.0 / 3.0, seed=3, n_modes=32).numpy()
    parity(x, 1e-3, 1, 0, 1.5, 4.0)
for order in range(6):
    for shape in [(37, 50, 148), (45, 70, 136)]:
        x = synth.grf(shape, 5.0 / 3.0, seed=order, n_modes=32).numpy()
        parity(x, 1e-3, order % 2, order, 1.25, 2.0)
for stride in (2, 8, 64, 256):
    x = synth.grf((40, 41, 90), 5.0 / 3.0, seed=5, n_modes=32).numpy()
    parity(x, 1e-3, 1, 2, 1.5, 4.0, stride)
for order in (0, 1):
    x = synth.grf((300, 517), 3.0, seed=9, n_modes=32).numpy()
    parity(x, 1e-3, 1, order, 1.5, 4.0)

x = torch.from_numpy(synth.grf((48, 48, 48), 5.0 / 3.0, seed=11, n_modes=32).numpy()).cuda()
opts = q.make_tune_opts(block=16, rate=0.2, n_orders=6)
for metric, target in ((q.METRIC_MAXERR, float("nan")), (q.METRIC_PSNR, float("nan")),
                       (q.METRIC_PSNR, 70.0), (q.METRIC_SSIM, 0.999),
                       (q.METRIC_AC, float("nan"))):
    q.tune(x, 1e-3, metric, target, opts)
    out["cases"] += 1
y = x + 1e-3 * torch.randn_like(x)
m = q.compute_metrics(x, y, 1.0, 7, 2)
q.error_autocorr(x, y, 3)
fields = [torch.from_numpy(synth.grf(s, 5.0 / 3.0, seed=i, n_modes=16).numpy()).cuda()
          for i, s in enumerate([(40, 33, 70), (1, 200, 301), (64, 64, 64)])]
blobs = q.compress_batch(fields, 1e-3)
for b in blobs:
    b.free()
out["cases"] += 1
out["record"] = q.debug_bounds(reset=True)
print(json.dumps(out))
"""


def test_bounds_checking_build_records_nothing():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2310_14133_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, QOZ_LIBRARY=lib, PYTHONPATH=ROOT)
    p = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    res = json.loads(p.stdout.strip().splitlines()[-1])
    assert res["cases"] >= 30
    assert res["record"] == 0, f"index check failed: line {(res['record'] >> 40) & 0x7fffff}, " \
                               f"index {res['record'] & 0xffffffffff}"


def test_product_build_has_no_bounds_record():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2310_14133_gb300 as q
    with pytest.raises(q.QozError) as ei:
        q.debug_bounds()
    assert ei.value.status == 6
