"""Seeded synthetic inputs: modified stochastic block model graphs (m-SBM).

This package is the one module shared by the CUDA path's tests/bench and by the
CPU oracle.  It draws graphs only; it holds none of the clustering method's
arithmetic (no Laplacian, no projection, no eigensolver).

The m-SBM follows Appendix B.2 of Wang, Lu, Davidson and Bai, "Scalable
Spectral Clustering with Group Fairness Constraints" (AISTATS 2023):
vertices carry a planted cluster and a group; an undirected edge between two
distinct vertices is a Bernoulli draw whose probability depends only on
whether the endpoints share a cluster and whether they share a group
(eq. p-msbm), and the adjacency has no self loops (eq. w-msbm).
"""
from .generator import (
    Graph,
    cell_sizes_equal,
    cell_sizes_from_proportions,
    category_probabilities,
    sample_msbm,
    gaussian_edge_weights,
    graph_from_dense,
    random_constraints,
    random_weighted_graph,
)
from . import configs

__all__ = [
    "Graph",
    "cell_sizes_equal",
    "cell_sizes_from_proportions",
    "category_probabilities",
    "sample_msbm",
    "gaussian_edge_weights",
    "graph_from_dense",
    "random_weighted_graph",
    "random_constraints",
    "configs",
]
