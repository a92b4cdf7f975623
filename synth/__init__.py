"""Seeded synthetic WCSP / Bayesian-network / DCOP instances.

This package only draws random problem instances (variables, domains, scopes and
cost tables).  It holds none of the elimination arithmetic: both the CPU oracle
(test infrastructure) and the CUDA library consume the instances it produces.
"""
from .generators import (  # noqa: F401
    Instance,
    grid_wcsp,
    er_wcsp,
    bayes_net_mpe,
    bn_prefix,
    dcop_random,
    dcop_stream,
    random_small,
    paper_example,
    scale_free_wcsp,
    random_network_wcsp,
    disjoint_union,
    grid_mrf,
    ising_ring,
    coloring,
    with_evidence,
    config_instance,
    TOP_K,
)
