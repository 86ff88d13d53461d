"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the CPU oracle.

This package holds no arithmetic of the method itself (no basis ranking, no
matrix elements, no H*v): only lattices (bond lists), couplings, interaction
term lists, counter-based random start vectors and the named workloads.  Both
``oracle/`` and ``paper_2307_13222_gb300`` read its outputs; neither imports
the other.
"""
from .lattice import chain, ladder, square, random_regular_graph, splitmix64_stream, uniform_couplings
from .terms import heisenberg_terms, xxz_terms, hubbard_terms, TERM_KINDS
from .rng import philox4x32_10, philox_uniform53, philox_gaussian, random_vectors, bootstrap_picks
from . import configs

__all__ = [
    "chain", "ladder", "square", "random_regular_graph", "splitmix64_stream", "uniform_couplings",
    "heisenberg_terms", "xxz_terms", "hubbard_terms", "TERM_KINDS",
    "philox4x32_10", "philox_uniform53", "philox_gaussian", "random_vectors", "bootstrap_picks", "configs",
]
