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


def test_oversized_extents_are_refused_before_any_device_call():
    # the validation runs on the host before the first CUDA call: extents
    # whose product reaches 2^32, or wraps around 64 bits, give
    # QOZ_EUNSUPPORTED (the field pointer is never dereferenced)
    import ctypes as C
    from paper_2310_14133_gb300 import _binding as b
    lib = b.lib()
    out = C.c_void_p()
    fake = C.c_void_p(256)
    for dims, nd in (((1 << 22, 1 << 22, 1 << 22), 3), ((1 << 32, 1, 1), 3),
                     ((65536, 65536, 1), 3), ((1 << 40, 1 << 30, 0), 2),
                     ((3, 1 << 62, 4), 3)):
        s = b.Shape()
        s.ndims = nd
        for i, v in enumerate(dims):
            s.dims[i] = v
        st = lib.qoz_compress(fake, s, 1e-3, None, None, None, C.byref(out))
        assert st == 6, (dims, st)
        assert not out.value


def test_binding_checks_buffers_before_the_library():
    # sizes and host buffers are checked in the binding, so a wrong buffer
    # raises instead of letting the library write past its end
    import pytest
    import torch
    import paper_2310_14133_gb300 as q
    from paper_2310_14133_gb300 import _binding as b
    with pytest.raises(ValueError):
        q.deserialize(torch.zeros(64, dtype=torch.uint8)[::2])       # not contiguous
    with pytest.raises(ValueError):
        q.deserialize(torch.zeros(16, dtype=torch.float32))          # not bytes
    with pytest.raises(ValueError):
        b._same_points(torch.zeros(7), 8, "out")
    b._same_points(torch.zeros(2, 4), 8, "out")
    with pytest.raises(ValueError):
        b._host_bytes(torch.zeros(8, dtype=torch.int16), "out")
    assert b._host_bytes(torch.zeros(8, dtype=torch.uint8), "out").value


def test_parameter_builders_refuse_values_they_cannot_hold():
    # per-level entries are bytes: out-of-range values are refused instead of
    # wrapping into a valid one; validity itself (order < 6, ...) is the
    # library's check and still reaches it
    import pytest
    import paper_2310_14133_gb300 as q
    for bad in (256, -1, 300):
        with pytest.raises(ValueError):
            q.make_params(3, order=bad)
        with pytest.raises(ValueError):
            q.make_params(3, interp=[1, 1, bad])
    assert q.make_params(3, order=6).order[0] == 6
    with pytest.raises(ValueError):
        q.make_tune_opts(alphas=[1.0] * 9)
    with pytest.raises(ValueError):
        q.make_tune_opts(betas=[2.0] * 9)
    o = q.make_tune_opts(alphas=[1.0, 1.5], betas=[2.0])
    assert o.n_alpha == 2 and o.n_beta == 1 and o.alphas[1] == 1.5


def test_batch_bounds_per_field():
    import pytest
    from paper_2310_14133_gb300 import _binding as b
    assert b._per_field(1e-3, 3) == [1e-3] * 3
    assert b._per_field([1e-3, 2e-3], 2) == [1e-3, 2e-3]
    with pytest.raises(ValueError):
        b._per_field([1e-3, 2e-3], 3)
