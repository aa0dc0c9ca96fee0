"""GB300 (sm_103a) implementation of the Wedge hot path (arXiv 1903.07754).

The engine lives in libwedge.so (C ABI, include/wedge.h); ``wedge`` is its
ctypes binding.  Importing this package does not load CUDA.
"""
from .wedge import (  # noqa: F401
    BFS, CC, PR, SSSP, Graph, WedgeError, load, wedge_default_opts, wedge_frontier_transform,
    wedge_get_trace, wedge_graph_copy_edge_index, wedge_graph_create, wedge_graph_destroy,
    wedge_graph_get_info, wedge_graph_get_tuning, wedge_graph_set_tuning, wedge_kernel_launches, wedge_last_error, wedge_pull_iterate, wedge_run_bfs,
    wedge_run_cc, wedge_run_pr, wedge_run_sssp, wedge_version, wedge_mlp_forward, wedge_mlp_forward_bf16,
    wedge_mlp_loss_grad, wedge_mlp_adam, wedge_set_cost_model, wedge_trace_candidates, wedge_run_bfs_batch,
)
