"""Brute-force census of every 4-vertex subset (tiny graphs only, n <= 40).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is the plain definition of the counted quantity (Sec. 3, Problem 1, and
Fig. 1): for each of the C(n, 4) vertex subsets S, classify the induced
subgraph G[S] by its edge count and sorted degree sequence.  The six
connected classes are the paper's graphlets g1..g6; the other five classes
(empty, one edge, two adjacent edges, two disjoint edges, triangle plus an
isolated vertex) are disconnected and only serve the check that all eleven
classes together account for every one of the C(n, 4) subsets.
"""
from __future__ import annotations

import itertools

# (edge count, sorted degrees) -> class name
_CLASSES = {
    (0, (0, 0, 0, 0)): "empty",
    (1, (0, 0, 1, 1)): "edge",
    (2, (0, 1, 1, 2)): "wedge+isolated",
    (2, (1, 1, 1, 1)): "two-edges",
    (3, (0, 2, 2, 2)): "triangle+isolated",
    (3, (1, 1, 2, 2)): "g1",   # 3-path
    (3, (1, 1, 1, 3)): "g2",   # 3-star
    (4, (2, 2, 2, 2)): "g3",   # 4-cycle
    (4, (1, 2, 2, 3)): "g4",   # tailed triangle
    (5, (2, 2, 3, 3)): "g5",   # diamond
    (6, (3, 3, 3, 3)): "g6",   # 4-clique
}
CONNECTED = ("g1", "g2", "g3", "g4", "g5", "g6")
ALL_CLASSES = tuple(sorted(set(_CLASSES.values())))


def census(n: int, edges) -> dict[str, int]:
    """Histogram of the 11 induced 4-vertex classes over all C(n,4) subsets."""
    if n > 40:
        raise ValueError("brute force is for n <= 40")
    adj = [[False] * n for _ in range(n)]
    for a, b in edges:
        if a == b:
            raise ValueError("self-loop")
        adj[a][b] = adj[b][a] = True
    hist = {c: 0 for c in ALL_CLASSES}
    for s in itertools.combinations(range(n), 4):
        deg = [0, 0, 0, 0]
        k = 0
        for i in range(4):
            for j in range(i + 1, 4):
                if adj[s[i]][s[j]]:
                    k += 1
                    deg[i] += 1
                    deg[j] += 1
        hist[_CLASSES[(k, tuple(sorted(deg)))]] += 1
    return hist


def graphlet_counts(n: int, edges) -> list[int]:
    """[g1, g2, g3, g4, g5, g6] by brute force."""
    h = census(n, edges)
    return [h[c] for c in CONNECTED]


def census3(n: int, edges) -> dict[str, int]:
    """Histogram of the induced 3-vertex classes over all C(n,3) subsets:
    'empty', 'edge', 'path' (2 edges, the open wedge), 'triangle'."""
    if n > 60:
        raise ValueError("brute force is for n <= 60")
    adj = [[False] * n for _ in range(n)]
    for a, b in edges:
        adj[a][b] = adj[b][a] = True
    names = ("empty", "edge", "path", "triangle")
    hist = {k: 0 for k in names}
    for a, b, c in itertools.combinations(range(n), 3):
        hist[names[adj[a][b] + adj[a][c] + adj[b][c]]] += 1
    return hist


def graphlet3_counts(n: int, edges) -> list[int]:
    """[induced 2-paths, triangles] by the census."""
    h = census3(n, edges)
    return [h["path"], h["triangle"]]


def vertex_census(n: int, edges) -> list[list[int]]:
    """Per vertex, the number of induced connected 4-vertex graphlets
    [g1..g6] that contain it: every 4-subset adds its class to each of its
    four vertices (n <= 40)."""
    if n > 40:
        raise ValueError("brute force is for n <= 40")
    adj = [[False] * n for _ in range(n)]
    for a, b in edges:
        adj[a][b] = adj[b][a] = True
    idx = {c: i for i, c in enumerate(CONNECTED)}
    out = [[0] * 6 for _ in range(n)]
    for s in itertools.combinations(range(n), 4):
        deg = [0, 0, 0, 0]
        k = 0
        for i in range(4):
            for j in range(i + 1, 4):
                if adj[s[i]][s[j]]:
                    k += 1
                    deg[i] += 1
                    deg[j] += 1
        c = _CLASSES[(k, tuple(sorted(deg)))]
        if c in idx:
            for v in s:
                out[v][idx[c]] += 1
    return out


# orbit of a vertex inside each connected induced 4-vertex graph, by its
# degree there (the paw's two degree-2 corners share an orbit; its degree-2
# vertex set holds no tail): orbits 4..14 in the usual numbering of
# 4-vertex graphlet orbits
def _orbit(cls: str, deg: list[int], i: int) -> int:
    d = deg[i]
    if cls == "g1":
        return 4 if d == 1 else 5
    if cls == "g2":
        return 6 if d == 1 else 7
    if cls == "g3":
        return 8
    if cls == "g4":
        return {1: 9, 2: 10, 3: 11}[d]
    if cls == "g5":
        return 12 if d == 2 else 13
    return 14


def vertex_orbit_census(n: int, edges) -> list[list[int]]:
    """Per vertex, how many induced connected 4-vertex graphlets hold it in
    each orbit 4..14 (11 columns), over all 4-subsets (n <= 40)."""
    if n > 40:
        raise ValueError("brute force is for n <= 40")
    adj = [[False] * n for _ in range(n)]
    for a, b in edges:
        adj[a][b] = adj[b][a] = True
    out = [[0] * 11 for _ in range(n)]
    for s in itertools.combinations(range(n), 4):
        deg = [0, 0, 0, 0]
        k = 0
        for i in range(4):
            for j in range(i + 1, 4):
                if adj[s[i]][s[j]]:
                    k += 1
                    deg[i] += 1
                    deg[j] += 1
        c = _CLASSES[(k, tuple(sorted(deg)))]
        if c in CONNECTED:
            for i, v in enumerate(s):
                out[v][_orbit(c, deg, i) - 4] += 1
    return out


# edge orbit (0..9) of edge {a, b} inside each connected induced 4-vertex
# graph, by the degrees of its endpoints there: 3-path end, middle; 3-star;
# 4-cycle; tailed triangle tail, triangle edge opposite the attachment,
# triangle edge at the attachment; diamond outer edge, chord; 4-clique
def _edge_orbit(cls: str, deg: list[int], a: int, b: int) -> int:
    lo, hi = sorted((deg[a], deg[b]))
    if cls == "g1":
        return 0 if lo == 1 else 1
    if cls == "g2":
        return 2
    if cls == "g3":
        return 3
    if cls == "g4":
        return {(1, 3): 4, (2, 2): 5, (2, 3): 6}[(lo, hi)]
    if cls == "g5":
        return 8 if (lo, hi) == (3, 3) else 7
    return 9


def edge_orbit_census(n: int, edges):
    """Per edge (u < v, sorted), how many induced connected 4-vertex
    graphlets hold it in each edge orbit 0..9, over all 4-subsets (n <= 40).
    Returns (sorted edge list, list of 10-entry rows)."""
    if n > 40:
        raise ValueError("brute force is for n <= 40")
    adj = [[False] * n for _ in range(n)]
    for a, b in edges:
        adj[a][b] = adj[b][a] = True
    keys = sorted({(min(a, b), max(a, b)) for a, b in edges})
    row = {e: [0] * 10 for e in keys}
    for s in itertools.combinations(range(n), 4):
        deg = [0, 0, 0, 0]
        present = []
        for i in range(4):
            for j in range(i + 1, 4):
                if adj[s[i]][s[j]]:
                    deg[i] += 1
                    deg[j] += 1
                    present.append((i, j))
        c = _CLASSES[(len(present), tuple(sorted(deg)))]
        if c in CONNECTED:
            for i, j in present:
                row[(s[i], s[j])][_edge_orbit(c, deg, i, j)] += 1
    return keys, [row[e] for e in keys]
