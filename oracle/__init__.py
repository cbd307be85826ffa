"""QoZ oracle: Python access to the plain C++ CPU restatement of the method.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this package; the product path
(the CUDA library and its binding) never does, and the two share no code.

`build()` compiles qoz_oracle.cpp, qoz_oracle_tune.cpp, qoz_oracle_learn.cpp and
qoz_oracle_entropy.cpp with
-O2 -ffp-contract=off (no fused multiply-add, so binary32 arithmetic rounds
after every operation, as the CUDA side does with explicit _rn intrinsics).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["qoz_oracle.cpp", "qoz_oracle_tune.cpp", "qoz_oracle_learn.cpp",
            "qoz_oracle_entropy.cpp"]
_lib = None

MAX_LEVELS = 8
METRIC_MAXERR, METRIC_PSNR, METRIC_SSIM, METRIC_AC = 0, 1, 2, 3


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_HERE, "qoz_oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in deps):
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-fPIC",
           "-shared", "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("anchor_stride", C.c_int32),
                ("interp", C.c_uint8 * MAX_LEVELS),
                ("order", C.c_uint8 * MAX_LEVELS),
                ("alpha", C.c_double),
                ("beta", C.c_double)]


class LevelStats(C.Structure):
    _fields_ = [("l1", C.c_double * MAX_LEVELS), ("cnt", C.c_int64 * MAX_LEVELS)]


class TuneOpts(C.Structure):
    _fields_ = [("block", C.c_int32), ("rate", C.c_double), ("n_orders", C.c_int32),
                ("n_alpha", C.c_int32), ("alphas", C.c_double * 8),
                ("n_beta", C.c_int32), ("betas", C.c_double * 8),
                ("ssim_win", C.c_int32), ("ssim_step", C.c_int32),
                ("anchor_stride", C.c_int32)]


class Trial(C.Structure):
    _fields_ = [("bits", C.c_double), ("B", C.c_double), ("npts", C.c_int64),
                ("n_unpred", C.c_int64), ("n_anchors", C.c_int64),
                ("max_err", C.c_double), ("sse", C.c_double),
                ("ssim_sum", C.c_double), ("ssim_n", C.c_int64), ("stats", LevelStats),
                ("ac", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("params", Params), ("e", C.c_double), ("B", C.c_double), ("M", C.c_double),
                ("n_trials", C.c_int32), ("n_blocks", C.c_int32),
                ("n_sampled_points", C.c_int64), ("alg1_score", C.c_double * MAX_LEVELS)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        i64, f64, i32 = C.c_int64, C.c_double, C.c_int
        sig = {
            "orc_value_range": (i64, [P, i64, P, P]),
            "orc_level_bounds": (None, [f64, f64, f64, i32, P]),
            "orc_order_axes": (None, [i32, i32, P]),
            "orc_compress": (i32, [P, i32, P, f64, P, i32, P, P, P, P, P, P, i64, P, P]),
            "orc_decompress": (i32, [P, i32, P, f64, P, P, P, P, i64, P]),
            "orc_anchor_count": (i64, [i32, P, i32]),
            "orc_histogram": (None, [P, i32, P, i32, P]),
            "orc_huffman_bits": (C.c_uint64, [P, i32]),
            "orc_huffman_lengths": (i32, [P, i32, P]),
            "orc_canonical_codes": (None, [P, i32, P]),
            "orc_huffman_encode": (i64, [P, i64, i32, P, P, P, P, i64]),
            "orc_huffman_decode": (i32, [P, P, i64, i32, P, P, i32, P]),
            "orc_huffman_subruns": (i32, [P, i64, i32, P, P]),
            "orc_estimate_bits": (f64, [P, i64, i64]),
            "orc_max_abs_err": (f64, [P, P, i64]),
            "orc_mse": (f64, [P, P, i64]),
            "orc_autocorr": (f64, [P, P, i64, i64]),
            "orc_autocorr_blocks": (f64, [P, P, i64, i64]),
            "orc_psnr": (f64, [P, P, i64, f64]),
            "orc_ssim": (f64, [P, P, i32, P, i32, i32, f64, P, P]),
            "orc_sample_blocks": (i64, [i32, P, i32, f64, P, i64, P, P]),
            "orc_block_trial": (i32, [P, i32, P, P, i64, P, P, f64, i32, i32, i32, f64, P]),
            "orc_trial_metric": (f64, [P, i32, f64]),
            "orc_table1": (i32, [f64, f64, f64, f64, f64, f64, P]),
            "orc_tune": (i32, [P, i32, P, f64, f64, i32, f64, P, P]),
            "orc_ab_candidate": (None, [P, i32, P, P]),
            "orc_select_fixed": (i32, [i32, P, P, i32, RETRIAL_FN, P]),
            "orc_target_scale": (f64, [f64, f64]),
            "orc_target_rate": (f64, [f64, f64, f64, f64, f64]),
            "orc_secant_step": (i32, [f64, f64, f64, f64, f64, f64, f64, P]),
            "orc_target_pick": (i32, [i32, P, P, f64, f64]),
            "orc_features": (i32, [P, i32, P, f64, f64, P, i64, P, P]),
            "orc_mlp_forward": (None, [P, P, P, P, i64, P]),
            "orc_mlp_loss_grad": (f64, [P, P, P, P, P, i64, P]),
            "orc_adam_step": (None, [P, P, P, P, i64, i64, f64, f64, f64, f64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims(shape) -> np.ndarray:
    return np.ascontiguousarray(np.array(shape, dtype=np.int64))


def _level_value(v, l):
    """Per-level value: a scalar applies to every level; a list gives level
    l+1 its entry l, its last entry repeating above its length."""
    if isinstance(v, (list, tuple)):
        return v[min(l, len(v) - 1)]
    return v


def make_params(ndims: int, interp=1, order=0, alpha=1.0, beta=1.0, anchor_stride=None) -> Params:
    """Params with the same interpolator/order on every level, or per-level
    lists (index l-1 for level l)."""
    p = Params()
    p.anchor_stride = anchor_stride or (32 if ndims == 3 else 64)
    for l in range(MAX_LEVELS):
        p.interp[l] = _level_value(interp, l)
        p.order[l] = _level_value(order, l)
    p.alpha, p.beta = float(alpha), float(beta)
    return p


def value_range(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float32)
    mn, mx = C.c_float(), C.c_float()
    cnt = lib().orc_value_range(_ptr(x), x.size, C.byref(mn), C.byref(mx))
    return mn.value, mx.value, cnt


def level_bounds(e: float, alpha: float, beta: float, L: int):
    out = np.zeros(L, dtype=np.float64)
    lib().orc_level_bounds(e, alpha, beta, L, _ptr(out))
    return out


def order_axes(ndims: int, order: int):
    out = np.zeros(ndims, dtype=np.int32)
    lib().orc_order_axes(ndims, order, _ptr(out))
    return tuple(int(v) for v in out)


def anchor_count(shape, anchor_stride: int) -> int:
    d = _dims(shape)
    return int(lib().orc_anchor_count(len(shape), _ptr(d), anchor_stride))


def compress(x: np.ndarray, e: float, params: Params, stop_level: int = 1, want_recon=True):
    x = np.ascontiguousarray(x, dtype=np.float32)
    d = _dims(x.shape)
    n = x.size
    codes = np.zeros(x.shape, dtype=np.uint16)
    recon = np.zeros(x.shape, dtype=np.float32) if want_recon else None
    na_max = anchor_count(x.shape, params.anchor_stride)
    anchors = np.zeros(na_max, dtype=np.float32)
    na = C.c_int64()
    nu = C.c_int64()
    stats = LevelStats()
    cap = max(1024, n // 64)
    while True:
        uidx = np.zeros(cap, dtype=np.int64)
        uval = np.zeros(cap, dtype=np.float32)
        rc = lib().orc_compress(_ptr(x), x.ndim, _ptr(d), float(e), C.byref(params), stop_level,
                                _ptr(codes), _ptr(recon) if want_recon else None,
                                _ptr(anchors), C.byref(na), _ptr(uidx), _ptr(uval), cap,
                                C.byref(nu), C.byref(stats))
        if rc != 0:
            raise ValueError(f"orc_compress rejected its arguments (status {rc})")
        if nu.value <= cap:
            break
        cap = nu.value
    return {
        "codes": codes, "recon": recon, "anchors": anchors[:na.value],
        "unpred_idx": uidx[:nu.value].copy(), "unpred_val": uval[:nu.value].copy(),
        "l1": np.array(stats.l1[:]), "cnt": np.array(stats.cnt[:]),
    }


def decompress(codes: np.ndarray, e: float, params: Params, anchors, unpred_idx, unpred_val):
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    d = _dims(codes.shape)
    out = np.zeros(codes.shape, dtype=np.float32)
    anchors = np.ascontiguousarray(anchors, dtype=np.float32)
    ui = np.ascontiguousarray(unpred_idx, dtype=np.int64)
    uv = np.ascontiguousarray(unpred_val, dtype=np.float32)
    rc = lib().orc_decompress(_ptr(codes), codes.ndim, _ptr(d), float(e), C.byref(params),
                              _ptr(anchors), _ptr(ui), _ptr(uv), ui.size, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_decompress failed (status {rc})")
    return out


def histogram(codes: np.ndarray, anchor_stride: int) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    d = _dims(codes.shape)
    h = np.zeros(65536, dtype=np.uint64)
    lib().orc_histogram(_ptr(codes), codes.ndim, _ptr(d), anchor_stride, _ptr(h))
    return h


def huffman_bits(hist) -> int:
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    return int(lib().orc_huffman_bits(_ptr(h), h.size))


def huffman_lengths(hist):
    """Code length per symbol (uint8 array) and the longest length."""
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    ln = np.zeros(h.size, dtype=np.uint8)
    mx = int(lib().orc_huffman_lengths(_ptr(h), h.size, _ptr(ln)))
    return ln, mx


def canonical_codes(lengths):
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.zeros(ln.size, dtype=np.uint64)
    lib().orc_canonical_codes(_ptr(ln), ln.size, _ptr(code))
    return code


ENTROPY_CHUNK = 4096


def entropy_chunk(n: int) -> int:
    """The stream's chunk size for n codes (a layout the paper leaves open;
    this project's reading): the largest of 4096, 2048, 1024, 512 and 256
    codes that still gives at least 8192 chunks, else 256."""
    c = ENTROPY_CHUNK
    while c > 256 and -(-n // c) < 8192:
        c //= 2
    return c


def huffman_encode(symbols, lengths, codes, chunk: int | None = None):
    """(words uint32, offs uint64) of the chunked MSB-first stream; chunk
    None takes entropy_chunk of the symbol count."""
    s = np.ascontiguousarray(symbols, dtype=np.uint16).ravel()
    chunk = entropy_chunk(s.size) if chunk is None else int(chunk)
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    cd = np.ascontiguousarray(codes, dtype=np.uint64)
    nch = (s.size + chunk - 1) // chunk
    offs = np.zeros(nch + 1, dtype=np.uint64)
    cap = int(np.sum(ln[s].astype(np.int64)) // 32) + nch + 1
    words = np.zeros(max(cap, 1), dtype=np.uint32)
    w = int(lib().orc_huffman_encode(_ptr(s), s.size, chunk, _ptr(ln), _ptr(cd), _ptr(offs),
                                     _ptr(words), words.size))
    if w < 0:
        raise ValueError(f"encode failed ({w})")
    return words[:w].copy(), offs


def huffman_subruns(symbols, lengths, chunk: int | None = None):
    """The stream's sub-run table (uint16, n_chunks x (S - 1) entries in chunk
    order; empty when S = 1): the coded length in bits of each 512-code run
    of a chunk but its last.  chunk None takes entropy_chunk."""
    s = np.ascontiguousarray(symbols, dtype=np.uint16).ravel()
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    chunk = entropy_chunk(s.size) if chunk is None else int(chunk)
    S = chunk // 512 if chunk >= 1024 else 1
    nch = (s.size + chunk - 1) // chunk
    sub = np.zeros(max(nch * (S - 1), 1), dtype=np.uint16)
    r = int(lib().orc_huffman_subruns(_ptr(s), s.size, chunk, _ptr(ln), _ptr(sub)))
    if r < 0:
        raise ValueError("a symbol without a code")
    return sub[:nch * (S - 1)].copy()


def huffman_decode(words, offs, n: int, lengths, codes, chunk: int | None = None):
    chunk = entropy_chunk(n) if chunk is None else int(chunk)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    o = np.ascontiguousarray(offs, dtype=np.uint64)
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    cd = np.ascontiguousarray(codes, dtype=np.uint64)
    out = np.zeros(n, dtype=np.uint16)
    st = int(lib().orc_huffman_decode(_ptr(w), _ptr(o), n, chunk, _ptr(ln), _ptr(cd), ln.size,
                                      _ptr(out)))
    if st != 0:
        raise ValueError("decode failed")
    return out


def autocorr(a, b, lag: int = 1) -> float:
    """Eq. (ac) of the errors b - a over the flattened arrays."""
    a = np.ascontiguousarray(a, dtype=np.float32).ravel()
    b = np.ascontiguousarray(b, dtype=np.float32).ravel()
    return float(lib().orc_autocorr(_ptr(a), _ptr(b), a.size, lag))


def autocorr_blocks(errors, sizes, lag: int = 1) -> float:
    """Eq. (ac) over errors cut into consecutive blocks of the given sizes:
    pairs inside a block, mean and variance over all."""
    e = np.ascontiguousarray(errors, dtype=np.float64).ravel()
    st = np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64))]).astype(np.int64)
    assert st[-1] == e.size
    return float(lib().orc_autocorr_blocks(_ptr(e), _ptr(st), st.size - 1, lag))


def estimate_bits(hist, n_unpred: int, n_anchors: int) -> float:
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    assert h.size == 65536
    return float(lib().orc_estimate_bits(_ptr(h), n_unpred, n_anchors))


def max_abs_err(a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(lib().orc_max_abs_err(_ptr(a), _ptr(b), a.size))


def mse(a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(lib().orc_mse(_ptr(a), _ptr(b), a.size))


def psnr(a, b, vrange: float) -> float:
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    return float(lib().orc_psnr(_ptr(a), _ptr(b), a.size, vrange))


def ssim(a, b, vrange: float, win: int = 7, step: int = 2):
    """Returns (mean, n_windows, sum)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    d = _dims(a.shape)
    nw = C.c_int64()
    s = C.c_double()
    m = lib().orc_ssim(_ptr(a), _ptr(b), a.ndim, _ptr(d), win, step, vrange, C.byref(nw),
                       C.byref(s))
    return float(m), int(nw.value), float(s.value)


def sample_blocks(shape, block: int, rate: float):
    d = _dims(shape)
    bd = np.ones(3, dtype=np.int64)
    S = C.c_int64()
    nb = lib().orc_sample_blocks(len(shape), _ptr(d), block, rate, None, 0, _ptr(bd),
                                 C.byref(S))
    org = np.zeros((max(nb, 1), 3), dtype=np.int64)
    lib().orc_sample_blocks(len(shape), _ptr(d), block, rate, _ptr(org), nb, _ptr(bd),
                            C.byref(S))
    return org[:nb], tuple(int(v) for v in bd[:len(shape)]), int(S.value)


def block_trial(x, origins, block_dims, params: Params, e: float, stop_level=1,
                ssim_win=0, ssim_step=2, vrange=1.0) -> Trial:
    x = np.ascontiguousarray(x, dtype=np.float32)
    d = _dims(x.shape)
    org = np.ascontiguousarray(origins, dtype=np.int64)
    bd = np.ones(3, dtype=np.int64)
    bd[:len(block_dims)] = block_dims
    t = Trial()
    rc = lib().orc_block_trial(_ptr(x), x.ndim, _ptr(d), _ptr(org), org.shape[0], _ptr(bd),
                               C.byref(params), float(e), stop_level, ssim_win, ssim_step,
                               float(vrange), C.byref(t))
    if rc != 0:
        raise ValueError("orc_block_trial failed")
    return t


def trial_metric(t: Trial, metric: int, vrange: float) -> float:
    return float(lib().orc_trial_metric(C.byref(t), metric, vrange))


def table1(b1, m1, b2, m2, b2p=float("nan"), m2p=float("nan")):
    """Returns (decision, second_scale): decision 0 keep I, 1 take II, -1 needs
    II at second_scale * e."""
    sc = C.c_double(0.0)
    r = lib().orc_table1(b1, m1, b2, m2, b2p, m2p, C.byref(sc))
    return int(r), float(sc.value)


RETRIAL_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_double,
                         C.POINTER(C.c_double), C.POINTER(C.c_double))


def ab_candidate(opts, k):
    """(alpha, beta) of candidate k of the tuner's search."""
    a, b = C.c_double(), C.c_double()
    lib().orc_ab_candidate(C.byref(opts), int(k), C.byref(a), C.byref(b))
    return float(a.value), float(b.value)


def select_fixed(B, M, maxerr_mode=False, retrial=None):
    """Sec. 6.3.2 keep-best over candidates in order.  retrial(k, scale) ->
    (B', M') supplies solution II's second point when Table I asks for it.
    Returns the kept index."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)

    def cb(_ctx, k, scale, pb, pm):
        if retrial is None:
            return 1
        b, m = retrial(int(k), float(scale))
        pb[0], pm[0] = float(b), float(m)
        return 0

    fn = RETRIAL_FN(cb)
    r = lib().orc_select_fixed(len(B), _ptr(B), _ptr(M), 1 if maxerr_mode else 0, fn, None)
    if r < 0:
        raise ValueError("orc_select_fixed failed")
    return int(r)


def target_scale(M, target):
    return float(lib().orc_target_scale(float(M), float(target)))


def target_rate(B, M, B2, M2, target):
    return float(lib().orc_target_rate(float(B), float(M), float(B2), float(M2), float(target)))


def secant_step(ea, ma, eb, mb, target, e0, e_user):
    """Returns the next bound of the target mode's secant, or None (no step)."""
    en = C.c_double(0.0)
    r = lib().orc_secant_step(float(ea), float(ma), float(eb), float(mb), float(target),
                              float(e0), float(e_user), C.byref(en))
    return float(en.value) if r else None


def target_pick(e, M, target, e_user):
    e = np.ascontiguousarray(e, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    return int(lib().orc_target_pick(len(e), _ptr(e), _ptr(M), float(target), float(e_user)))


def make_tune_opts(ndims: int, block=None, rate=None, n_orders=None, alphas=None, betas=None,
                   ssim_win=7, ssim_step=2, anchor_stride=None) -> TuneOpts:
    """Defaults are the paper's (Sec. 7.1.4, Sec. 6.3.1): 3D b=16, r=0.5 %,
    s=32; 2D b=64, r=1 %, s=64; alpha {1,1.25,1.5,1.75,2}, beta {1.5,2,3,4};
    two dimension orders (increasing and decreasing)."""
    o = TuneOpts()
    o.block = block or (16 if ndims == 3 else 64)
    o.rate = rate or (0.005 if ndims == 3 else 0.01)
    o.n_orders = n_orders or 2
    al = alphas or [1.0, 1.25, 1.5, 1.75, 2.0]
    be = betas or [1.5, 2.0, 3.0, 4.0]
    o.n_alpha = len(al)
    o.n_beta = len(be)
    for i, v in enumerate(al):
        o.alphas[i] = v
    for i, v in enumerate(be):
        o.betas[i] = v
    o.ssim_win, o.ssim_step = ssim_win, ssim_step
    o.anchor_stride = anchor_stride or (32 if ndims == 3 else 64)
    return o


def tune(x, e_user: float, vrange: float, metric: int, target=float("nan"), opts=None):
    x = np.ascontiguousarray(x, dtype=np.float32)
    d = _dims(x.shape)
    opts = opts or make_tune_opts(x.ndim)
    r = TuneResult()
    rc = lib().orc_tune(_ptr(x), x.ndim, _ptr(d), float(e_user), float(vrange), metric,
                        float(target), C.byref(opts), C.byref(r))
    if rc != 0:
        raise ValueError("orc_tune failed")
    return r


# ------------------------------------------------------------ learned tuner
NFEAT, NHID, NOUT = 64, 128, 16
NPARAM = NHID * NFEAT + NHID + NHID * NHID + NHID + NOUT * NHID + NOUT
HEADS = ((0, 2), (2, 6), (8, 5), (13, 3))   # (offset, length): interp, order, alpha, beta


def features(x, rel_eb: float, vrange: float, block: int, rate: float):
    """The 64 features of the blocks sampled with (block, rate)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    d = _dims(x.shape)
    org, bd, _ = sample_blocks(x.shape, block, rate)
    org = np.ascontiguousarray(org, dtype=np.int64)
    bdv = np.ones(3, dtype=np.int64)
    bdv[:len(bd)] = bd
    out = np.zeros(NFEAT, dtype=np.float64)
    rc = lib().orc_features(_ptr(x), x.ndim, _ptr(d), float(rel_eb), float(vrange), _ptr(org),
                            len(org), _ptr(bdv), _ptr(out))
    if rc != 0:
        raise ValueError("orc_features failed")
    return out


def features_blocks(x, rel_eb: float, vrange: float, origins, block_dims):
    """Features over explicit blocks (origins [nb, 3], block_dims per axis)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    d = _dims(x.shape)
    org = np.ascontiguousarray(origins, dtype=np.int64).reshape(-1, 3)
    bdv = np.ones(3, dtype=np.int64)
    bdv[:len(block_dims)] = block_dims
    out = np.zeros(NFEAT, dtype=np.float64)
    rc = lib().orc_features(_ptr(x), x.ndim, _ptr(d), float(rel_eb), float(vrange), _ptr(org),
                            len(org), _ptr(bdv), _ptr(out))
    if rc != 0:
        raise ValueError("orc_features failed")
    return out


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n
    return a


def mlp_forward(params, mean, sd, X):
    X = _f64(X).reshape(-1, NFEAT)
    out = np.zeros((X.shape[0], NOUT), dtype=np.float64)
    lib().orc_mlp_forward(_ptr(_f64(params, NPARAM)), _ptr(_f64(mean, NFEAT)),
                          _ptr(_f64(sd, NFEAT)), _ptr(X), X.shape[0], _ptr(out))
    return out


def mlp_loss_grad(params, mean, sd, X, labels, want_grad=True):
    X = _f64(X).reshape(-1, NFEAT)
    lab = np.ascontiguousarray(labels, dtype=np.int32).reshape(-1, 4)
    g = np.zeros(NPARAM, dtype=np.float64) if want_grad else None
    loss = lib().orc_mlp_loss_grad(_ptr(_f64(params, NPARAM)), _ptr(_f64(mean, NFEAT)),
                                   _ptr(_f64(sd, NFEAT)), _ptr(X), _ptr(lab), X.shape[0],
                                   _ptr(g) if want_grad else None)
    return float(loss), g


def adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on params, m, v (float64 arrays)."""
    lib().orc_adam_step(_ptr(params), _ptr(_f64(grad)), _ptr(m), _ptr(v), params.size, int(t),
                        float(lr), float(beta1), float(beta2), float(eps))

