"""libfsort: GB300-native compressed radix sort (arXiv 2605.10390 hot path).

Python binding over the C ABI declared in ``include/fsort.h``.  Every function
here only marshals arguments (tensors -> device pointers, the current torch
stream -> cudaStream_t) and raises :class:`FsortError` on a non-OK status; the
sort itself runs in the CUDA kernels of ``libfsort.so``.  There is no CPU or
PyTorch fallback: if the library is missing, every call raises.

Low-level names mirror the C ABI (``fsort_plan_create``, ``fsort_sort_pairs``,
...).  :class:`Plan` is a small convenience wrapper for torch tensors.
"""
from ._binding import (  # noqa: F401
    FSORT_FLAG_GRAPH,
    FSORT_FLAG_HOST_IO,
    FSORT_FLAG_LEARNED,
    FSORT_LEARN_CELLS,
    FSORT_LEARN_MAX_HEAVY,
    FSORT_MLP_PARAMS,
    FsortLearnedOpts,
    FsortLearnedStats,
    fsort_learned_bucket_ids,
    fsort_learned_fit,
    fsort_learned_get_model,
    fsort_learned_get_stats,
    fsort_learned_set_model,
    fsort_mlp_forward,
    fsort_mlp_grad,
    FsortBatchConfig,
    FsortSegment,
    fsort_batch_autotune,
    fsort_batch_get_config,
    fsort_batch_set_config,
    fsort_sort_batch,
    FsortError,
    FsortKernelTime,
    KERNEL_KINDS,
    FsortPlanDesc,
    FsortPlanInfo,
    Plan,
    STATUS,
    fsort_exclusive_scan,
    fsort_expand,
    fsort_histogram,
    fsort_plan_create,
    fsort_plan_describe,
    fsort_plan_device_flags,
    fsort_plan_destroy,
    fsort_plan_set_timing,
    fsort_plan_sync,
    fsort_plan_timing_report,
    fsort_scatter_pass,
    fsort_scatter_pass_noalloc,
    FSORT_NOALLOC_MAX_KEYS,
    fsort_sort_pairs,
    fsort_sort_pairs_host,
    fsort_sort_pairs_out,
    fsort_status_string,
    fsort_version,
    lib_path,
    load_library,
)
