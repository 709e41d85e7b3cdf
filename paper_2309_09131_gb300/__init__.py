"""GB300-native (sm_103a) FLYCOO spMTTKRP with dynamic tensor remapping.

The computation lives in the CUDA library ``_lib/libflycoo.so`` (C ABI in
``include/flycoo.h``); this package is its ctypes binding plus a thin owning
wrapper.  PyTorch supplies device memory and streams only.
"""
from ._native import (  # noqa: F401
    BF16,
    F32,
    FlycooError,
    flycoo_all_modes_host,
    flycoo_cp_als,
    flycoo_cp_als_step,
    flycoo_cpopt_grad,
    flycoo_debug_fail_alloc_after,
    flycoo_debug_set_wait_limit,
    flycoo_create,
    flycoo_destroy,
    flycoo_export_layout,
    flycoo_export_next,
    flycoo_export_partition,
    flycoo_export_schedule,
    flycoo_export_tile_order,
    flycoo_get_info,
    flycoo_last_error,
    flycoo_mttkrp_adjoint,
    flycoo_plan_create,
    flycoo_plan_destroy,
    flycoo_plan_get,
    flycoo_remap,
    flycoo_spmttkrp,
    flycoo_spmttkrp_static_scratch,
    flycoo_sync,
    flycoo_timing_enable,
    flycoo_timing_read,
    make_params,
)
from ._native import (  # noqa: F401
    PLAN_G,
    PLAN_K4_ITEMS,
    PLAN_K4_NLIGHT,
    PLAN_K4_ORDER,
    PLAN_SHARD_BIN_PTR,
    PLAN_SHARD_ITEMS,
    PLAN_SHARD_PTR,
    PLAN_SHARD_SS,
    PLAN_SS_BIN_PTR,
    PLAN_SS_ITEMS,
    PLAN_SS_SHARD_PTR,
    PLAN_TILE_BIN_PTR_512,
    PLAN_TILE_BIN_PTR_1024,
    PLAN_TILES_512,
    PLAN_TILES_1024,
    PLAN_SEG_SS,
    PLAN_SS_SEG_PTR,
    ORDER_KEY,
    ORDER_MORTON,
    SCHEDULE_BLOCK_CYCLIC,
    SCHEDULE_LPT,
)
from .flycoo import FlycooTensor  # noqa: F401
from .autograd import CPOPTLoss, SpMTTKRP, cpopt_loss, spmttkrp  # noqa: F401
