"""GB300-native recursive density-matrix purification (libpurify).

The compute path is the CUDA shared library ``libpurify.so`` (sm_103a); this
package only marshals arguments to its C ABI.  Build it with
``paper_1101_0265_gb300.build.build()``.
"""
from ._lib import (  # noqa: F401
    BRANCH_RULES, Batch, ERR_BOUNDS, batch_footprint, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_INVALID_ARG, ERR_NOT_CONVERGED,
    ERR_INTERNAL, ERR_OOM, ERR_STATE, ERR_UNSUPPORTED, EXPORTED, LIB_PATH, OK, PRECISIONS, SCHEMES, Purifier,
    PurifyError, k_digit_product_f64, k_gershgorin_f64, k_gershgorin_f64_noalloc,
    GERSHGORIN_NOALLOC_MAX_N, k_lanczos_f64, k_step_f64, k_symm_product_f64, load, schedule,
    strerror, tridiag_eig, tuned_shape,
)
