"""swdb: Smith-Waterman/Gotoh protein database search on one GB300 GPU.

The compute path is libswdb.so (hand-written CUDA for sm_103a behind a C
ABI, declared in include/swdb.h).  This package is a thin ctypes binding
with the same entry-point names; it only marshals arguments.  There is no
CPU fallback: if the library is missing, every call raises.
"""
from .binding import (  # noqa: F401
    ALIGNMENT_DTYPE,
    HIT_DTYPE,
    SW_ALIGN_GLOBAL,
    SW_ALIGN_LOCAL,
    SW_ALIGN_OVERLAP,
    SW_ALIGN_SEMIGLOBAL,
    SW_OP_D,
    SW_OP_I,
    SW_OP_M,
    SW_FLAG_GRAPH,
    SW_MODE_AUTO,
    SW_MODE_BATCHED,
    SW_MODE_PLAIN,
    SW_PREC_AUTO,
    SW_PREC_I16,
    SW_PREC_I32,
    SwError,
    Database,
    ShardedDatabase,
    load_library,
    library_path,
    sw_align,
    sw_align_ops_capacity,
    sw_db_free,
    sw_db_get_info,
    sw_db_get_tuning,
    sw_db_load,
    sw_db_set_tuning,
    sw_hits_merge,
    sw_last_error,
    sw_probe_alu_rate,
    sw_probe_wait_timeout,
    sw_search,
    sw_search_no_alloc,
    sw_search_workspace_size,
    sw_scores_scatter,
    sw_shard_plan,
    sw_top_k,
    sw_version,
)
