"""GB300 batch-dynamic 4-node graphlet counting (FDGC / IGC, arXiv 2308.14493).

The compute path is the CUDA library ``libgc.so`` behind the C ABI in
``include/gc.h``; ``gc`` is its ctypes binding.  Importing this package does
not load the library; the first call does, and fails loudly if it cannot.
"""
from .gc import (  # noqa: F401
    GRAPHLETS,
    GCError,
    Graph,
    Server,
    gc_apply_batch,
    gc_apply_batch_device,
    gc_apply_batches,
    gc_apply_batches_device,
    gc_batch_stats,
    gc_close,
    gc_count_batch,
    gc_count_batch_device,
    gc_delete_vertices,
    gc_count_static,
    gc_count_static_noalloc,
    gc_device_bytes,
    gc_get_tuning,
    gc_set_tuning,
    gc_autotune,
    gc_batch_bytes,
    gc_trim,
    gc_server_open,
    gc_server_submit,
    gc_server_wait,
    gc_server_drain,
    gc_server_counters,
    gc_server_close,
    gc_counts,
    gc_counts3,
    gc_export_csr,
    gc_last_error,
    gc_num_edges,
    gc_open,
    library_path,
    load,
)
