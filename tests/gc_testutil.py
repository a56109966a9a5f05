"""Small helpers shared by the tests (graph building, golden parsing, BFS)."""
from __future__ import annotations

import os
from collections import deque

import numpy as np

from synth import gen

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def csr_from_edges(n, edges):
    keys = np.array(sorted({(min(a, b) << 32) | max(a, b) for a, b in edges}), dtype=np.uint64)
    return gen.csr_from_keys(n, keys)


def edges_from_csr(row_ptr, col):
    rp = np.asarray(row_ptr, dtype=np.int64)
    out = []
    for u in range(rp.size - 1):
        for v in col[rp[u]:rp[u + 1]]:
            if u < v:
                out.append((u, int(v)))
    return out


def random_graph(rng, n, p):
    return [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]


def load_closed_forms():
    """Parse ``golden/closed_forms.txt`` -> list of (name, n, edges, expect)."""
    out = []
    cur = None
    with open(os.path.join(GOLDEN_DIR, "closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "graph":
                cur = dict(name=tok[1], n=int(tok[2]), edges=[], expect=None)
                out.append(cur)
            elif tok[0] == "edges":
                cur["edges"] = [tuple(int(x) for x in t.split("-")) for t in tok[1:]]
            elif tok[0] == "expect":
                cur["expect"] = [int(x) for x in tok[1:]]
    return [(c["name"], c["n"], c["edges"], c["expect"]) for c in out]


def bfs_region(n, adj_rows, sources, hops):
    """Vertices within ``hops`` of any source (plain queue walk)."""
    dist = {}
    q = deque()
    for s in sources:
        if s not in dist:
            dist[s] = 0
            q.append(s)
    while q:
        x = q.popleft()
        if dist[x] >= hops:
            continue
        for y in adj_rows[x]:
            if y not in dist:
                dist[y] = dist[x] + 1
                q.append(y)
    return sorted(dist)


def rows_of(row_ptr, col):
    rp = np.asarray(row_ptr, dtype=np.int64)
    return [list(map(int, col[rp[u]:rp[u + 1]])) for u in range(rp.size - 1)]
