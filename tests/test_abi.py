"""The C-ABI library builds, loads and exports every entry point that
include/qoz.h declares (no compute call: this runs without a GPU)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "qoz.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(qoz_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("qoz_compress", "qoz_decompress", "qoz_value_range", "qoz_compute_metrics",
                 "qoz_blob_serialize", "qoz_blob_deserialize", "qoz_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2310_14133_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_marshals_without_gpu():
    import paper_2310_14133_gb300 as q
    p = q.make_params(3, interp=[0, 1, 1], order=[5, 0, 2], alpha=1.25, beta=3)
    assert list(p.interp[:3]) == [0, 1, 1] and p.order[0] == 5 and p.beta == 3.0
    # an invalid call fails loudly through the status code, never falls back
    import torch
    x = torch.zeros(4)
    try:
        q.compress(x, 1e-3)
    except ValueError as e:
        assert "CUDA" in str(e)
    else:
        raise AssertionError("a CPU tensor must be rejected")
