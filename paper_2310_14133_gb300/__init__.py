"""GB300 (sm_103a) implementation of the QoZ compressor's data path.

The compute runs in the CUDA library libqoz.so (C ABI, include/qoz.h); this
package only marshals arguments to it.  PyTorch supplies device memory and
the current CUDA stream.  Importing the package fails loudly when the
library has not been built: there is no CPU fallback.

Typical use, with x a contiguous float32 CUDA tensor of 2 or 3 dimensions:

    import paper_2310_14133_gb300 as q
    opts = q.make_tune_opts(block=32, rate=0.005, n_orders=6)
    rep = q.tune(x, 1e-3, q.METRIC_PSNR, float("nan"), opts)   # Sec. 6 tuner
    blob = q.compress_abs(x, rep.abs_eb, rep.params)          # Sec. 5 predictor
    buf = blob.serialize()            # host uint8: header + Huffman-coded codes
    y = q.decompress(q.deserialize(buf))
    m = q.compute_metrics(x, y, rep.vmax - rep.vmin, 7, 2)    # max error, PSNR, SSIM, AC

Calls take an optional `stream` (a torch.cuda.Stream) and otherwise run on
torch's current stream.  Blobs own device memory until `free()` (or garbage
collection).  Many fields of fixed shapes go through one `Batch` plan; a
trained `Model` proposes the tuner's choices (`tune_learned`,
`tune_learned_verified`).
"""

from ._binding import (  # noqa: F401
    METRIC_AC,
    METRIC_MAXERR,
    METRIC_PSNR,
    METRIC_SSIM,
    STAGE_DLEVEL,
    STAGE_HIST,
    STAGE_LEVEL,
    STAGE_RANGE,
    STAGE_METRICS,
    STAGE_SETUP,
    STAGE_TUNE,
    STAGE_FEATURES,
    STAGE_FORWARD,
    BATCH_AUTOTUNE,
    BATCH_NO_GRAPH,
    Batch,
    BatchInfo,
    Blob,
    HEADS,
    MLP_PARAMS,
    Model,
    NFEATURES,
    QozError,
    Shape,
    compress,
    compress_abs,
    compress_batch,
    compute_metrics,
    debug_bounds,
    decompress,
    deserialize,
    error_autocorr,
    features,
    lib,
    library_path,
    make_params,
    make_tune_opts,
    profile_enable,
    profile_read,
    tune,
    tune_learned,
    tune_learned_verified,
    tune_verify,
    value_range,
)
