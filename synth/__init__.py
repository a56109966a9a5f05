"""Seeded synthetic inputs: random graphs and update-batch streams.

This package holds only random sampling (splitmix64 counters, Erdos-Renyi and
Chung-Lu graphs, batch streams).  It contains none of the graphlet-counting
arithmetic, so both the CPU oracle and the CUDA path may draw their inputs from
it without sharing any part of the method.
"""
from .gen import (  # noqa: F401
    splitmix64,
    uniform01,
    er_graph,
    chung_lu_graph,
    csr_from_keys,
    keys_from_csr,
    random_batch,
    batch_stream,
    WORKLOADS,
    workload_graph,
)
