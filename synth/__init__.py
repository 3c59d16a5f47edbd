"""Seeded synthetic inputs for the Euler-tour path.

This package only draws random trees, graphs and query batches. It holds none
of the method's arithmetic, so both the CPU oracle tests and the CUDA path can
use it without sharing any computation.
"""

from .generators import (  # noqa: F401
    tree_parent,
    lca_queries,
    easy_graph,
    hard_graph,
    ba_tree,
    batched_instances,
    serving_stream,
    make_tree,
    make_graph,
)
