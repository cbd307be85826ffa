"""GB300 (sm_103a) implementation of the QoZ compressor's data path.

The compute runs in the CUDA library libqoz.so (C ABI, include/qoz.h); this
package only marshals arguments to it.  PyTorch supplies device memory and
the current CUDA stream.  Importing the package fails loudly when the
library has not been built: there is no CPU fallback.
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
