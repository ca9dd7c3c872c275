"""Seeded synthetic graph generators shared by the oracle tests, the CUDA tests and bench.py.

This module holds no arithmetic of the annealing method itself: it only draws graphs.
Every draw comes from a counter-based splitmix64 stream keyed by (seed, stream, index), so a
graph is a pure function of its parameters and does not depend on numpy's RNG versions.
"""
from .graphs import (  # noqa: F401
    CSRGraph, splitmix64, uniform01, erdos_renyi, torus2d, barabasi_albert,
    random_geometric, er_batch, batch_union, from_edges, path_graph, star_graph,
)
