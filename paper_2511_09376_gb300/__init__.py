"""GB300 (sm_103a) Background SHAP for decision-tree ensembles (WOODELF hot path).

Thin ctypes binding over the C ABI in ``include/woodelf.h``; the names mirror it:
``ctx_create``, ``load_ensemble``, ``set_background``, ``explain``,
``expected_value``, ``global_attribution`` and the ``debug_*`` inspectors.  The
binding only marshals arguments -- every step of the computation runs in the CUDA
library.  If the library has not been built, importing the binding raises.
"""
from ._binding import (  # noqa: F401
    BF16X3,
    BF16X6,
    Batch,
    batch_autotune,
    batch_create,
    background_counts,
    background_counts_size,
    batch_explain,
    batch_tile_rows,
    FP32,
    TF32X3,
    Context,
    Ensemble,
    Server,
    WdfError,
    ctx_create,
    debug_leaf_hist,
    debug_pair_table,
    ensemble_info,
    expected_value,
    explain,
    explain_interactions,
    set_background_counts,
    global_attribution,
    global_attribution_noalloc,
    launch_count,
    library_path,
    load_ensemble,
    server_create,
    server_poll,
    server_reset_stats,
    server_stats,
    server_submit,
    server_wait,
    set_background,
    set_covers,
    set_path_dependent,
    set_metric,
    version,
)
