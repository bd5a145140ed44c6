"""GB300 (sm_103a) Background SHAP for decision-tree ensembles (WOODELF hot path).

Thin ctypes binding over the C ABI in ``include/woodelf.h``; the names mirror it:
``ctx_create``, ``load_ensemble``, ``set_background``, ``explain``,
``expected_value``, ``global_attribution`` and the ``debug_*`` inspectors.  The
binding only marshals arguments -- every step of the computation runs in the CUDA
library.

The CUDA library is loaded on the first use of one of these names, not when the
package is imported, so that ``paper_2511_09376_gb300.synth`` (the seeded input
generator, which holds none of the method's arithmetic) can be imported without it.
If the library has not been built, that first use raises ImportError.
"""
from __future__ import annotations

_BINDING_NAMES = (
    "BF16X3", "BF16X6", "FP32", "TF32X3",
    "Batch", "Context", "Ensemble", "Server", "WdfError",
    "background_counts", "background_counts_size",
    "batch_autotune", "batch_create", "batch_explain", "batch_tile_rows",
    "ctx_create", "debug_contract_wait_limit", "debug_leaf_hist", "debug_pair_table",
    "ensemble_info", "expected_value", "explain", "explain_interactions", "explain_timing", "explain_timing_read",
    "global_attribution", "global_attribution_noalloc",
    "launch_count", "library_path", "load_ensemble",
    "server_create", "server_poll", "server_request_ms", "server_reset_stats", "server_stats", "server_submit", "server_wait",
    "set_background", "set_background_counts", "set_covers", "set_metric", "set_path_dependent",
    "version",
)

__all__ = list(_BINDING_NAMES)


def __getattr__(name):
    if name in _BINDING_NAMES:
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")


def __dir__():
    return sorted(set(globals()) | set(_BINDING_NAMES))
