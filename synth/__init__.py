"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This package holds input generators only: graphs (Barabasi-Albert, Holme-Kim,
R-MAT, small named graphs), uniformly random deletion sets, and the per-instance
draws of the batched workload.  It contains none of the method's arithmetic
(no fitness, no genetic operator, no Philox) and imports neither the CUDA
package nor the oracle.  Its random stream is SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), written
out in numpy so that a seed gives the same graph on every machine and numpy
version.
"""
from .rng import splitmix64, SplitMixStream
from .graphs import (
    Graph,
    ba_graph,
    hk_graph,
    rmat_graph,
    csr_from_edges,
    named_graph,
    er_graph,
    relabel,
    batched_instances,
)
from .populations import random_deletion_sets

__all__ = [
    "splitmix64",
    "SplitMixStream",
    "Graph",
    "ba_graph",
    "hk_graph",
    "rmat_graph",
    "csr_from_edges",
    "named_graph",
    "er_graph",
    "relabel",
    "batched_instances",
    "random_deletion_sets",
]
