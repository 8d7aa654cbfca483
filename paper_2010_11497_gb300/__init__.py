"""GB300-native Cluster-and-Conquer (C^2, arXiv 2010.11497) KNN-graph builder.

The compute lives in libc2.so (hand-written sm_103a CUDA kernels behind the
C ABI of include/c2.h); this package is its Python binding.
"""
from ._c2 import (C2Error, Model, ModelConfig, c2_autotune_report, c2_autotune_load, c2_autotune_save, Options, STRATEGY_AUTO, STRATEGY_MERGE, STRATEGY_TABLE32,  # noqa: F401
                  STRATEGY_MMA,
                  STRATEGY_TABLE64, c2_avg_sim, c2_bruteforce_knn, c2_build_knn_graph,
                  c2_build_knn_graph_host, c2_cluster_knn, c2_exact_counts, c2_goldfinger, c2_frh_cluster, c2_get_stats,
                  c2_get_status, c2_kernel_launches, c2_merge_topk,
                  c2_merge_topk_noalloc, c2_merge_topk_noalloc_max_slots, c2_minhash_keys,
                  c2_profile_enable, c2_profile_report, c2_reset_status, c2_status_string,
                  header_functions, lib, options, workspace, workspace_size,
                  workspace_size_host)
