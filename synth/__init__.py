"""Seeded synthetic workloads for the GNN-MPC real-time-iteration step.

This package only draws random numbers and lays out plain data (graphs,
weights, states, references, bounds, obstacles).  It holds none of the
method's arithmetic: no GNN evaluation, no Jacobians, no condensing, no QP.
Both the FP64 oracle and the CUDA path read their inputs from here, so the two
see bit-identical float32 inputs.
"""
from .workloads import (  # noqa: F401
    Workload,
    chain_edges,
    random_local_edges,
    gnn_layer_shapes,
    gnn_blob_size,
    make_gnn_blob,
    make_workload,
    small_chain,
    paper_chain,
    random_instance,
    CONFIGS,
)
