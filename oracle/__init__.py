"""CPU oracle for batch-dynamic 4-node graphlet counting.

TEST INFRASTRUCTURE ONLY.  Nothing in the library path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library.

* ``brute``  -- census of every 4-subset (n <= 40) and every 3-subset
  (n <= 60), the plain definitions.
* ``oracle`` -- plain single-threaded C (``gc_oracle.c``): literal and
  degree-oriented static counts, the 3-vertex counts, batch normalisation and
  one literal step of Algorithm 2 (FDGC); plain Python over adjacency sets
  for the eleven 4-vertex types, the per-vertex orbits and the per-edge
  orbits, each pinned against the census of every 4-subset.
"""
from . import brute  # noqa: F401
from .oracle import (  # noqa: F401
    ALL_TYPES,
    EDGE_ORBITS,
    GRAPHLETS,
    SUMS,
    OracleGraph,
    build,
    counts_all,
    counts_from_sums,
    edge_orbits,
    fdgc_step,
    normalize,
    static_counts,
    static_counts3,
    sums_literal,
    sums_oriented,
    vertex_counts,
    vertex_orbits,
)
