"""ctypes binding of libqoz.so: same names as the C ABI, argument marshalling
only.  Tensors must be CUDA tensors on the current device; the stream is
torch's current stream unless one is given."""

from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# QOZ_LIBRARY may name another build of the same library (the bounds-checking
# build of build.build(debug_bounds=True)); the default is the product build.
_LIB = os.environ.get("QOZ_LIBRARY") or os.path.join(_HERE, "_build", "libqoz.so")

MAX_LEVELS = 8
METRIC_MAXERR, METRIC_PSNR, METRIC_SSIM, METRIC_AC = 0, 1, 2, 3
STATUS = {0: "QOZ_OK", 1: "QOZ_EINVAL", 2: "QOZ_ENOMEM", 3: "QOZ_ECUDA", 4: "QOZ_ECORRUPT",
          5: "QOZ_ETIMEOUT", 6: "QOZ_EUNSUPPORTED"}


class QozError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Shape(C.Structure):
    _fields_ = [("ndims", C.c_int32), ("dims", C.c_int64 * 3)]


class Params(C.Structure):
    _fields_ = [("anchor_stride", C.c_int32), ("interp", C.c_uint8 * MAX_LEVELS),
                ("order", C.c_uint8 * MAX_LEVELS), ("alpha", C.c_double), ("beta", C.c_double)]


class BlobInfo(C.Structure):
    _fields_ = [("shape", Shape), ("params", Params), ("abs_eb", C.c_double),
                ("rel_eb", C.c_double), ("vmin", C.c_float), ("vmax", C.c_float),
                ("n_points", C.c_int64), ("n_anchors", C.c_int64),
                ("n_unpredictable", C.c_int64), ("est_bits", C.c_double),
                ("est_ratio", C.c_double)]


PROF_STAGES = 32
STAGE_RANGE, STAGE_SETUP, STAGE_LEVEL, STAGE_HIST, STAGE_FINAL = 0, 1, 2, 11, 12
STAGE_DLEVEL, STAGE_METRICS, STAGE_TUNE = 12, 21, 22
STAGE_FEATURES, STAGE_FORWARD = 23, 24


class StageTimes(C.Structure):
    _fields_ = [("ms", C.c_double * PROF_STAGES), ("calls", C.c_int64 * PROF_STAGES),
                ("launches", C.c_int64)]


def profile_enable(on: bool = True, stages=None):
    """Turns per-stage event timing on or off; `stages` (an iterable of stage
    ids) limits the timed stages, None times all of them."""
    mask = 0xFFFFFFFF if stages is None else sum(1 << int(i) for i in stages)
    _check(lib().qoz_profile_stages(mask))
    _check(lib().qoz_profile_enable(1 if on else 0))


def debug_bounds(reset: bool = True) -> int:
    """Record of the first index check that failed since the last reset (0:
    none).  Raises QozError (QOZ_EUNSUPPORTED) on the product build."""
    v = C.c_uint64()
    _check(lib().qoz_debug_bounds(C.byref(v), 1 if reset else 0))
    return v.value


def profile_read(reset: bool = False) -> StageTimes:
    t = StageTimes()
    _check(lib().qoz_profile_read(C.byref(t), 1 if reset else 0))
    return t


class TuneOpts(C.Structure):
    _fields_ = [("block", C.c_int32), ("rate", C.c_double), ("n_orders", C.c_int32),
                ("n_alpha", C.c_int32), ("alphas", C.c_double * 8),
                ("n_beta", C.c_int32), ("betas", C.c_double * 8),
                ("ssim_win", C.c_int32), ("ssim_step", C.c_int32),
                ("anchor_stride", C.c_int32)]


class TuneReport(C.Structure):
    _fields_ = [("params", Params), ("abs_eb", C.c_double), ("vmin", C.c_double),
                ("vmax", C.c_double), ("B", C.c_double), ("M", C.c_double),
                ("n_trials", C.c_int32), ("n_blocks", C.c_int32),
                ("n_sampled_points", C.c_int64), ("alg1_score", C.c_double * MAX_LEVELS)]


def make_tune_opts(block=0, rate=0.0, n_orders=0, alphas=None, betas=None, ssim_win=0,
                   ssim_step=0, anchor_stride=0) -> TuneOpts:
    """Zero / None fields take the library's defaults (the paper's)."""
    o = TuneOpts()
    for name, vals in (("alphas", alphas), ("betas", betas)):
        if len(vals or []) > 8:
            raise ValueError(f"at most 8 {name} (got {len(vals)})")
    o.block, o.rate, o.n_orders = block, rate, n_orders
    for i, v in enumerate(alphas or []):
        o.alphas[i] = v
    o.n_alpha = len(alphas or [])
    for i, v in enumerate(betas or []):
        o.betas[i] = v
    o.n_beta = len(betas or [])
    o.ssim_win, o.ssim_step, o.anchor_stride = ssim_win, ssim_step, anchor_stride
    return o


def tune(x: torch.Tensor, rel_eb: float, metric: int = 0, target: float = float("nan"),
         opts: TuneOpts | None = None, stream=None) -> TuneReport:
    rep = TuneReport()
    _check(lib().qoz_tune(_dev_ptr(x), _shape_of(x), float(rel_eb), int(metric), float(target),
                          C.byref(opts) if opts is not None else None, _stream(stream),
                          C.byref(rep)))
    return rep


class Metrics(C.Structure):
    _fields_ = [("max_abs_err", C.c_double), ("mse", C.c_double), ("psnr", C.c_double),
                ("ssim", C.c_double), ("ssim_windows", C.c_int64), ("ac", C.c_double)]


_lib = None


def library_path() -> str:
    return _LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise ImportError(
                f"{_LIB} is missing: build it with paper_2310_14133_gb300/build.py "
                "(or __graft_entry__.build()); there is no CPU fallback")
        _lib = C.CDLL(_LIB)
        P = C.c_void_p
        i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
        sig = {
            "qoz_last_error": (C.c_char_p, []),
            "qoz_value_range": (i32, [P, i64, P, P, P, P]),
            "qoz_value_range_noalloc": (i32, [P, i64, P, P, P]),
            "qoz_compress": (i32, [P, Shape, f64, P, P, P, P]),
            "qoz_compress_abs": (i32, [P, Shape, f64, P, P, P, P]),
            "qoz_decompress": (i32, [P, P, P]),
            "qoz_blob_get_info": (i32, [P, P]),
            "qoz_blob_arrays": (i32, [P, P, P, P, P, P, P]),
            "qoz_blob_copy_arrays": (i32, [P, P, P, P, P, P]),
            "qoz_blob_histogram": (i32, [P, P, P]),
            "qoz_blob_check": (i32, [P, P]),
            "qoz_blob_serialize": (i32, [P, P, C.c_size_t, P, P]),
            "qoz_blob_serialize_async": (i32, [P, P, C.c_size_t, P, P]),
            "qoz_blob_serialize_bound": (i32, [P, P]),
            "qoz_blob_deserialize": (i32, [P, C.c_size_t, P, P]),
            "qoz_blob_free": (None, [P]),
            "qoz_compute_metrics": (i32, [P, P, Shape, f64, i32, i32, P, P]),
            "qoz_error_autocorr": (i32, [P, P, i64, i64, P, P]),
            "qoz_profile_enable": (i32, [i32]),
            "qoz_profile_stages": (i32, [C.c_uint32]),
            "qoz_debug_bounds": (i32, [P, i32]),
            "qoz_tune": (i32, [P, Shape, f64, i32, f64, P, P, P]),
            "qoz_profile_read": (i32, [P, i32]),
            "qoz_batch_create": (i32, [P, i32, P, C.c_uint32, P]),
            "qoz_batch_compress": (i32, [P, P, P, i32, P, P]),
            "qoz_batch_get_info": (i32, [P, P]),
            "qoz_batch_free": (None, [P]),
            "qoz_compress_batch": (i32, [P, P, i32, f64, P, P, P]),
            "qoz_features": (i32, [P, Shape, f64, P, P, P, P]),
            "qoz_model_create": (i32, [C.c_uint64, P]),
            "qoz_model_set": (i32, [P, P, P, P]),
            "qoz_model_get": (i32, [P, P, P, P]),
            "qoz_model_forward": (i32, [P, P, i64, P, P]),
            "qoz_model_gradient": (i32, [P, P, P, i64, P, P, P]),
            "qoz_model_train_step": (i32, [P, P, P, i64, C.c_float, P, P]),
            "qoz_model_free": (None, [P]),
            "qoz_tune_learned": (i32, [P, Shape, f64, i32, f64, P, P, P, P]),
            "qoz_tune_learned_verified": (i32, [P, Shape, f64, i32, f64, P, P, P, P]),
            "qoz_tune_verify": (i32, [P, Shape, f64, i32, f64, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _check(status: int):
    if status != 0:
        raise QozError(status, lib().qoz_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _shape_of(t: torch.Tensor) -> Shape:
    if t.dim() not in (2, 3):
        raise QozError(1, f"fields must be 2D or 3D (got {t.dim()} dimensions)")
    s = Shape()
    s.ndims = t.dim()
    for i, d in enumerate(t.shape):
        s.dims[i] = int(d)
    return s


def _shape_tuple(dims) -> Shape:
    if len(dims) not in (2, 3):
        raise QozError(1, f"fields must be 2D or 3D (got {len(dims)} dimensions)")
    s = Shape()
    s.ndims = len(dims)
    for i, d in enumerate(dims):
        s.dims[i] = int(d)
    return s


def _dev_ptr(t: torch.Tensor, dtype=torch.float32):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {dtype} tensor")
    return C.c_void_p(t.data_ptr())


def _host_bytes(t: torch.Tensor, what: str):
    """A host buffer the library writes or reads as raw bytes."""
    if t.is_cuda or t.dtype != torch.uint8 or not t.is_contiguous():
        raise ValueError(f"{what} must be a contiguous host uint8 tensor")
    return C.c_void_p(t.data_ptr())


def _same_points(t: torch.Tensor, n: int, what: str):
    if t.numel() != n:
        raise ValueError(f"{what} holds {t.numel()} values, the field {n}")


def _u8(v, what: str) -> int:
    """A per-level entry of the parameter block (one byte).  Values that do
    not fit are refused here rather than wrapped; which values are valid is
    the library's check."""
    v = int(v)
    if not 0 <= v <= 255:
        raise ValueError(f"{what} {v} does not fit the parameter block")
    return v


def _level_value(v, l):
    """Per-level value: a scalar applies to every level; a list gives level
    l+1 its entry l, its last entry repeating above its length."""
    if isinstance(v, (list, tuple)):
        return v[min(l, len(v) - 1)]
    return v


def make_params(ndims: int, interp=1, order=0, alpha=1.0, beta=1.0, anchor_stride=0) -> Params:
    """Same interpolator/order on every level, or per-level lists (index l-1
    is level l)."""
    p = Params()
    p.anchor_stride = anchor_stride
    for l in range(MAX_LEVELS):
        p.interp[l] = _u8(_level_value(interp, l), "interp")
        p.order[l] = _u8(_level_value(order, l), "order")
    p.alpha, p.beta = float(alpha), float(beta)
    return p


def value_range(x: torch.Tensor, stream=None):
    mn, mx, cnt = C.c_float(), C.c_float(), C.c_int64()
    _check(lib().qoz_value_range(_dev_ptr(x), x.numel(), C.byref(mn), C.byref(mx),
                                 C.byref(cnt), _stream(stream)))
    return mn.value, mx.value, cnt.value


class Blob:
    """A compressed field; owns its device memory until freed."""

    def __init__(self, handle: C.c_void_p, shape):
        self._h = handle
        self.shape = tuple(shape)

    @property
    def handle(self):
        return self._h

    def info(self) -> BlobInfo:
        inf = BlobInfo()
        _check(lib().qoz_blob_get_info(self._h, C.byref(inf)))
        return inf

    def arrays(self, stream=None):
        """Copies of (codes [shape] as int16 bit patterns of the uint16 codes,
        unpredictable indices int64, unpredictable values float32, anchors
        float32) as CUDA tensors."""
        inf = self.info()
        codes = torch.empty(self.shape, dtype=torch.int16, device="cuda")
        ui = torch.empty(inf.n_unpredictable, dtype=torch.int64, device="cuda")
        uv = torch.empty(inf.n_unpredictable, dtype=torch.float32, device="cuda")
        an = torch.empty(inf.n_anchors, dtype=torch.float32, device="cuda")
        _check(lib().qoz_blob_copy_arrays(self._h, C.c_void_p(codes.data_ptr()),
                                          C.c_void_p(ui.data_ptr()), C.c_void_p(uv.data_ptr()),
                                          C.c_void_p(an.data_ptr()), _stream(stream)))
        return codes, ui, uv, an

    def check(self, stream=None) -> None:
        """Raises QozError(QOZ_ECORRUPT) when the last decompression met a
        code-0 point without an unpredictable-list entry (synchronises)."""
        _check(lib().qoz_blob_check(self._h, _stream(stream)))

    def histogram(self, stream=None) -> torch.Tensor:
        h = torch.zeros(65536, dtype=torch.int32)
        _check(lib().qoz_blob_histogram(self._h, C.c_void_p(h.data_ptr()), _stream(stream)))
        return h.to(torch.int64)

    def serialize(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        used = C.c_size_t()
        _check(lib().qoz_blob_serialize(self._h, None, 0, C.byref(used), _stream(stream)))
        if out is None:
            out = torch.empty(used.value, dtype=torch.uint8, pin_memory=True)
        ptr = _host_bytes(out, "out")
        if out.numel() < used.value:
            raise ValueError("output buffer too small")
        _check(lib().qoz_blob_serialize(self._h, ptr, out.numel(), C.byref(used),
                                        _stream(stream)))
        return out[:used.value]

    def serialize_bound(self) -> int:
        """Upper bound on the serialized size (no device work)."""
        b = C.c_size_t()
        _check(lib().qoz_blob_serialize_bound(self._h, C.byref(b)))
        return b.value

    def serialize_async(self, out: torch.Tensor, stream=None) -> int:
        """Enqueues the serialized stream into `out` (pinned host uint8) on the
        stream; complete once the stream is synchronized.  Returns its size."""
        used = C.c_size_t()
        _check(lib().qoz_blob_serialize_async(self._h, _host_bytes(out, "out"), out.numel(),
                                              C.byref(used), _stream(stream)))
        return used.value

    def free(self):
        if self._h:
            lib().qoz_blob_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def compress(x: torch.Tensor, rel_eb: float, params: Params | None = None,
             recon: torch.Tensor | None = None, stream=None) -> Blob:
    h = C.c_void_p()
    if recon is not None:
        _same_points(recon, x.numel(), "recon")
    _check(lib().qoz_compress(_dev_ptr(x), _shape_of(x), float(rel_eb),
                              C.byref(params) if params is not None else None,
                              _dev_ptr(recon) if recon is not None else None,
                              _stream(stream), C.byref(h)))
    return Blob(h, x.shape)


def compress_abs(x: torch.Tensor, abs_eb: float, params: Params | None = None,
                 recon: torch.Tensor | None = None, stream=None) -> Blob:
    h = C.c_void_p()
    if recon is not None:
        _same_points(recon, x.numel(), "recon")
    _check(lib().qoz_compress_abs(_dev_ptr(x), _shape_of(x), float(abs_eb),
                                  C.byref(params) if params is not None else None,
                                  _dev_ptr(recon) if recon is not None else None,
                                  _stream(stream), C.byref(h)))
    return Blob(h, x.shape)


def decompress(blob: Blob, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(blob.shape, dtype=torch.float32, device="cuda")
    else:
        _same_points(out, math.prod(blob.shape), "out")
    _check(lib().qoz_decompress(blob.handle, _dev_ptr(out), _stream(stream)))
    return out


def deserialize(buf: torch.Tensor, stream=None) -> Blob:
    h = C.c_void_p()
    ptr = _host_bytes(buf, "buf")
    _check(lib().qoz_blob_deserialize(ptr, buf.numel(), _stream(stream), C.byref(h)))
    b = Blob(h, ())
    inf = b.info()
    b.shape = tuple(int(inf.shape.dims[i]) for i in range(inf.shape.ndims))
    return b


def compute_metrics(a: torch.Tensor, b: torch.Tensor, vrange: float, ssim_win: int = 0,
                    ssim_step: int = 2, stream=None) -> Metrics:
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    m = Metrics()
    _check(lib().qoz_compute_metrics(_dev_ptr(a), _dev_ptr(b), _shape_of(a), float(vrange),
                                     int(ssim_win), int(ssim_step), C.byref(m), _stream(stream)))
    return m


def error_autocorr(a: torch.Tensor, b: torch.Tensor, lag: int = 1, stream=None) -> float:
    """Eq. (ac) of the errors b - a at the given lag, flattened order."""
    if a.numel() != b.numel():
        raise ValueError("size mismatch")
    v = C.c_double()
    _check(lib().qoz_error_autocorr(_dev_ptr(a), _dev_ptr(b), a.numel(), int(lag), C.byref(v),
                                    _stream(stream)))
    return v.value


BATCH_AUTOTUNE = 1
BATCH_NO_GRAPH = 2


class BatchInfo(C.Structure):
    _fields_ = [("nfields", C.c_int32), ("n_groups", C.c_int32),
                ("launches_per_run", C.c_int32), ("graph", C.c_int32),
                ("autotuned", C.c_int32), ("level1_groups", C.c_int32),
                ("level1_variant", C.c_int32 * 16), ("level1_ms", (C.c_double * 4) * 16),
                ("ctas_per_run", C.c_int64)]


def _params_array(params, shapes):
    if params is None:
        return None
    if isinstance(params, Params):
        params = [params] * len(shapes)
    if len(params) != len(shapes):
        raise ValueError("one Params per field")
    return (Params * len(shapes))(*params)


def _per_field(eb, n: int):
    """One bound per field: a scalar applies to all n fields, a sequence must
    hold exactly n."""
    if isinstance(eb, (int, float)):
        return [float(eb)] * n
    ebs = [float(v) for v in eb]
    if len(ebs) != n:
        raise ValueError(f"{len(ebs)} bounds for {n} fields")
    return ebs


class Batch:
    """A batched-compression plan for a fixed list of field shapes."""

    def __init__(self, shapes, params=None, autotune: bool = False, graph: bool = True):
        self.shapes = [tuple(int(d) for d in s) for s in shapes]
        arr = (Shape * len(self.shapes))(*[_shape_tuple(s) for s in self.shapes])
        self._params = _params_array(params, self.shapes)
        flags = (BATCH_AUTOTUNE if autotune else 0) | (0 if graph else BATCH_NO_GRAPH)
        h = C.c_void_p()
        _check(lib().qoz_batch_create(arr, len(self.shapes), self._params, flags, C.byref(h)))
        self._h = h

    def compress(self, fields, eb, relative: bool = True, stream=None):
        """Blobs of the fields (CUDA float32 tensors of the plan's shapes);
        eb: one bound or one per field."""
        n = len(self.shapes)
        if len(fields) != n:
            raise ValueError("one field per plan shape")
        for f, s in zip(fields, self.shapes):
            if tuple(f.shape) != s:
                raise ValueError(f"field shape {tuple(f.shape)} != plan shape {s}")
        ptrs = (C.c_void_p * n)(*[_dev_ptr(f).value for f in fields])
        eba = (C.c_double * n)(*_per_field(eb, n))
        outs = (C.c_void_p * n)()
        _check(lib().qoz_batch_compress(self._h, ptrs, eba, 1 if relative else 0,
                                        _stream(stream), outs))
        return [Blob(C.c_void_p(outs[i]), self.shapes[i]) for i in range(n)]

    def info(self) -> BatchInfo:
        inf = BatchInfo()
        _check(lib().qoz_batch_get_info(self._h, C.byref(inf)))
        return inf

    def free(self):
        if self._h:
            lib().qoz_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def compress_batch(fields, rel_eb: float, params=None, stream=None):
    """One-shot batched compression with one relative bound."""
    shapes = [tuple(f.shape) for f in fields]
    n = len(fields)
    arr = (Shape * n)(*[_shape_tuple(s) for s in shapes])
    ptrs = (C.c_void_p * n)(*[_dev_ptr(f).value for f in fields])
    outs = (C.c_void_p * n)()
    _check(lib().qoz_compress_batch(ptrs, arr, n, float(rel_eb), _params_array(params, shapes),
                                    _stream(stream), outs))
    return [Blob(C.c_void_p(outs[i]), shapes[i]) for i in range(n)]


# ------------------------------------------------------------ learned tuner
NFEATURES = 64
MLP_PARAMS = 26896
HEADS = ((0, 2), (2, 6), (8, 5), (13, 3))   # (offset, length): interp, order, alpha, beta


def features(x: torch.Tensor, rel_eb: float, opts=None, stream=None, device_out=None):
    """The 64 features of the sampled blocks: float64 numpy array, or, with
    device_out (a CUDA float32 tensor of 64 values), written there only."""
    h = None
    if device_out is None:
        h = np.zeros(NFEATURES, dtype=np.float64)
    else:
        _same_points(device_out, NFEATURES, "device_out")
    _check(lib().qoz_features(_dev_ptr(x), _shape_of(x), float(rel_eb),
                              C.byref(opts) if opts is not None else None,
                              C.c_void_p(h.ctypes.data) if h is not None else None,
                              _dev_ptr(device_out) if device_out is not None else None,
                              _stream(stream)))
    return h


class Model:
    """The tuner network on the GPU (weights, normalisation, Adam state)."""

    def __init__(self, seed: int = 0):
        h = C.c_void_p()
        _check(lib().qoz_model_create(C.c_uint64(seed), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def set(self, params=None, mean=None, sd=None):
        def arr(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float32)
            if a.size != n:
                raise ValueError(f"expected {n} values, got {a.size}")
            return a
        p, m, s = arr(params, MLP_PARAMS), arr(mean, NFEATURES), arr(sd, NFEATURES)
        _check(lib().qoz_model_set(self._h, *(C.c_void_p(a.ctypes.data) if a is not None
                                              else None for a in (p, m, s))))

    def get(self):
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        m = np.zeros(NFEATURES, dtype=np.float32)
        s = np.zeros(NFEATURES, dtype=np.float32)
        _check(lib().qoz_model_get(self._h, C.c_void_p(p.ctypes.data), C.c_void_p(m.ctypes.data),
                                   C.c_void_p(s.ctypes.data)))
        return p, m, s

    def forward(self, feats: torch.Tensor, stream=None) -> torch.Tensor:
        feats = feats.reshape(-1, NFEATURES)
        out = torch.empty((feats.shape[0], 16), dtype=torch.float32, device="cuda")
        _check(lib().qoz_model_forward(self._h, _dev_ptr(feats), feats.shape[0], _dev_ptr(out),
                                       _stream(stream)))
        return out

    def gradient(self, feats: torch.Tensor, labels: torch.Tensor, stream=None):
        feats = feats.reshape(-1, NFEATURES)
        _same_points(labels, 4 * feats.shape[0], "labels (4 per feature row)")
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
        loss = C.c_float()
        _check(lib().qoz_model_gradient(self._h, _dev_ptr(feats), _dev_ptr(labels, torch.int32),
                                        feats.shape[0], _dev_ptr(g), C.byref(loss),
                                        _stream(stream)))
        return float(loss.value), g

    def train_step(self, feats: torch.Tensor, labels: torch.Tensor, lr: float, want_loss=False,
                   stream=None):
        feats = feats.reshape(-1, NFEATURES)
        _same_points(labels, 4 * feats.shape[0], "labels (4 per feature row)")
        loss = C.c_float()
        _check(lib().qoz_model_train_step(self._h, _dev_ptr(feats), _dev_ptr(labels, torch.int32),
                                          feats.shape[0], C.c_float(lr),
                                          C.byref(loss) if want_loss else None, _stream(stream)))
        return float(loss.value) if want_loss else None

    def save(self, path: str):
        p, m, s = self.get()
        np.savez(path, params=p, mean=m, sd=s)

    def load(self, path: str):
        d = np.load(path)
        self.set(d["params"], d["mean"], d["sd"])

    def free(self):
        if self._h:
            lib().qoz_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tune_learned(x: torch.Tensor, rel_eb: float, model: Model, metric: int = 0,
                 target: float = float("nan"), opts=None, stream=None):
    rep = TuneReport()
    _check(lib().qoz_tune_learned(_dev_ptr(x), _shape_of(x), float(rel_eb), int(metric),
                                  float(target), C.byref(opts) if opts is not None else None,
                                  model.handle, _stream(stream), C.byref(rep)))
    return rep


def tune_learned_verified(x: torch.Tensor, rel_eb: float, model: Model, metric: int = 0,
                          target: float = float("nan"), opts=None, stream=None):
    rep = TuneReport()
    _check(lib().qoz_tune_learned_verified(_dev_ptr(x), _shape_of(x), float(rel_eb), int(metric),
                                           float(target),
                                           C.byref(opts) if opts is not None else None,
                                           model.handle, _stream(stream), C.byref(rep)))
    return rep


def tune_verify(x: torch.Tensor, rel_eb: float, params: Params, metric: int = 0,
                target: float = float("nan"), opts=None, stream=None):
    rep = TuneReport()
    _check(lib().qoz_tune_verify(_dev_ptr(x), _shape_of(x), float(rel_eb), int(metric),
                                 float(target), C.byref(opts) if opts is not None else None,
                                 C.byref(params), _stream(stream), C.byref(rep)))
    return rep

