"""GB300-native BlockBP message-update engine (arxiv 2603.13304).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/bbp.h``); this package is its thin Python binding.  There is no
CPU fallback: using the engine without the built library raises.
"""
from ._lib import (  # noqa: F401
    BBPError, BF16, BOTTOM, KT_ABSORB, KT_JACOBI, KT_ORTH, KT_QR, KT_TC, FP32, FP64, KAGOME, LEFT, RIGHT, SQUARE, TF32, TOP, EXPORTS, lib,
    bbp_block_rdm, bbp_create_peps, bbp_destroy, bbp_energy_per_site, bbp_expect_local, bbp_footprint_bytes,
    bbp_get_message, bbp_core_pmps, bbp_core_plan_debug, bbp_core_expect, bbp_ite_bond, bbp_ite, bbp_info, bbp_init_messages, bbp_iterate, bbp_k_fuse, bbp_k_qr, bbp_k_svd_trunc,
    bbp_k_panel_cluster, bbp_k_panel_qr, bbp_k_svd_work_bytes_rand, bbp_k_svd_trunc_rand, bbp_k_fma_peak, bbp_set_hermitise, bbp_expect_product, bbp_bond_energies,
    bbp_k_svd_stats, bbp_k_svd_trunc_noalloc, bbp_k_svd_work_bytes, bbp_k_tc_absorb, bbp_k_tc_absorb_bytes,
    bbp_k_tc_gemm, bbp_k_tc_gemm_tile, bbp_autotune_record, bbp_autotune_run, bbp_autotune_load, bbp_autotune_info,
    bbp_autotune_clear, bbp_batch_single_launch, bbp_set_fuse_cache, bbp_share_workers, bbp_ktimer_read, bbp_ktimer_select, bbp_last_error, bbp_norm, bbp_partition_blocks, bbp_plan_debug, bbp_set_execution, bbp_set_options, bbp_set_power_iters, bbp_stats,
    use_default_allocator, use_torch_allocator, bbp_batch_iterate, bbp_job, make_job, bbp_job_footprint_bytes,
    bbp_server_create, bbp_server_submit, bbp_server_step, bbp_server_poll, bbp_server_take, bbp_server_destroy,
)
from .build import build  # noqa: F401
