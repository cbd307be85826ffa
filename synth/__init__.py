"""Seeded synthetic scientific fields: the inputs shared by the oracle and the
CUDA path.

This module holds no part of the compression method.  It stands in for the
paper's datasets (Table II: NYX 512^3, CESM-ATM 1800x3600, Miranda, Hurricane,
...), which are not available here, with fields of the same shapes and of the
same kind of structure:

* Gaussian random fields with a shell-integrated power spectrum E(k) ~ k^-p,
  built from M seeded random Fourier modes (directions uniform on the sphere
  or circle, |k| log-uniform in [1, n_ref/4] cycles per box, amplitude
  |k|^((1-p)/2) so that E(k) ~ k^-p under log-uniform sampling, phases
  uniform), scaled to standard deviation sigma;
* a linear trend, tanh fronts, zonal bands and Gaussian vortex tubes.

All random draws come from numpy's PCG64 seeded with the given seed; the
evaluation runs in torch on whichever device is asked for (CPU for small
test fields, the GPU for the large ones).  A test or benchmark generates a
field once and hands the same bytes to both sides.
"""

from .fields import (  # noqa: F401
    grf_trend_field,
    grf_fronts_field,
    mixed_batch_fields,
    training_field_spec,
    vortex_field,
    fronts,
    grf,
    linear_trend,
    vortex_tubes,
    zonal_bands,
)
