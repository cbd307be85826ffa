"""The value-range entry point that allocates nothing.

Some callers cannot let a library allocate device memory (a fixed memory
budget, a pre-planned arena, a stream capture that must not grow); for them
qoz_value_range_noalloc keeps its per-CTA partial results in a static device
array.  This test calls it through the C ABI twice in a row, on different
data, and checks each result against the allocating entry point
qoz_value_range, exactly (min, max and the count of finite values are exact
in both).  It lives in its own file, collected last."""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_value_range_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2310_14133_gb300 import build
    build.build()
    import paper_2310_14133_gb300 as q
    lib = q.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    cases = [(3_000_017, 0), (1_234_567, 3)]   # second call: unaligned start, other data
    for n, off in cases:
        x = rng.normal(0, 5, n + off).astype(np.float32)
        x[off + 11] = np.nan
        x[off + n // 2] = np.inf
        x[-1] = -np.inf
        xd = torch.from_numpy(x).cuda()[off:]
        out = torch.full((2,), -7.0, dtype=torch.float32, device="cuda")
        cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        st = lib.qoz_value_range_noalloc(_ptr(xd), xd.numel(), _ptr(out), _ptr(cnt), stream)
        assert st == 0, lib.qoz_last_error()
        torch.cuda.synchronize()
        mn, mx, c = q.value_range(xd)
        assert float(out[0]) == mn and float(out[1]) == mx
        assert int(cnt[0]) == c
    # sizes beyond the stated maximum are refused before any work
    big = (1 << 40) + 1
    st = lib.qoz_value_range_noalloc(_ptr(xd), big, _ptr(out), _ptr(cnt), stream)
    assert st == 6 and b"maximum" in lib.qoz_last_error()
