"""Seeded synthetic problem instances shared by the oracle and the CUDA path.

This package holds input generation only (graphs, couplings, fields and the
edge-colouring schedule).  It contains none of the annealer's arithmetic, so
both sides can consume the same instances without sharing method code.
"""
from .generators import (  # noqa: F401
    Instance,
    random_regular_graph,
    random_tree,
    edge_colouring,
    delta_edge_colouring,
    misra_gries_colouring,
    check_colouring,
    make_instance,
    make_tree_instance,
    make_batch,
    heavy_hex_graph,
    make_heavy_hex_instance,
    random_gate_inputs,
    BASE_SEED,
)
