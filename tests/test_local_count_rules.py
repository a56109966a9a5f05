"""The rules behind the per-vertex and per-edge count kernels, restated in
plain Python and checked on the CPU against the censuses of every 4-subset.

The kernels do not count copies directly as the oracle does: they take
closed forms of degrees, per-edge triangle counts t, per-vertex triangle
sums and s(x) = sum_{w in N(x)} (d_w - 1); they list each triangle and each
4-clique once in a total vertex order and credit its vertices or edges;
and they walk the 4-cycles from their highest vertex u, counting for each
opposite corner w the common lower neighbours c_w, then crediting each
wedge u-a-w with c_w - 1 (the cycles through it) and each corner pair with
C(c_w, 2).  This file pins those rules (not the kernels: the GPU parity
tests pin those) on random graphs, in a random vertex order, so that a
wrong credit or a wrong closed form fails here first.
"""
import itertools
import math

import numpy as np

from oracle import brute
from gc_testutil import random_graph


def _graph(n, edges):
    N = [set() for _ in range(n)]
    for a, b in edges:
        N[a].add(b)
        N[b].add(a)
    return N


def _pivot_c4(n, N, rank, c4_off=1):
    """4-cycles from their highest vertex u (in rank order): per wedge
    u-a-w (a, w below u) the credit c_w - 1, and per opposite corner the
    cycle count C(c_w, 2).  Returns (per-edge credit, per-vertex credit)."""
    edge = {}
    vert = [0] * n
    for u in range(n):
        low = [a for a in N[u] if rank[a] < rank[u]]
        c = {}
        for a in low:
            for w in N[a]:
                if rank[w] < rank[u]:
                    c[w] = c.get(w, 0) + 1
        for a in low:
            for w in N[a]:
                if rank[w] < rank[u] and c[w] > 1:
                    for e in ((min(u, a), max(u, a)), (min(a, w), max(a, w))):
                        edge[e] = edge.get(e, 0) + c[w] - c4_off
                    vert[a] += c[w] - c4_off
        for w, x in c.items():
            vert[w] += math.comb(x, 2)
            vert[u] += math.comb(x, 2)
    return edge, vert


def _cliques_and_triangles(n, N, rank):
    """Triangles and 4-cliques, each listed once in rank order."""
    order = sorted(range(n), key=lambda x: rank[x])
    tris, k4s = [], []
    for i, u in enumerate(order):
        up = [v for v in order[i + 1:] if v in N[u]]
        for a, b in itertools.combinations(up, 2):
            if b in N[a]:
                tris.append((u, a, b))
                for z in up:
                    if rank[z] > rank[b] and z in N[a] and z in N[b]:
                        k4s.append((u, a, b, z))
    return tris, k4s


def edge_rows_by_kernel_rules(n, edges, rank, opp_off=2, outer_off=2, c4_off=1):
    """The per-edge rows by the kernels' rules; the offsets are the
    constants of the opposite, diamond-outer and 4-cycle credits (the
    planted-mistake test changes them)."""
    N = _graph(n, edges)
    d = [len(x) for x in N]
    key = lambda a, b: (min(a, b), max(a, b))
    t = {key(a, b): len(N[a] & N[b]) for a, b in edges}
    tri = [sum(t[key(x, w)] for w in N[x]) // 2 for x in range(n)]
    s = [sum(d[w] - 1 for w in N[x]) for x in range(n)]
    opp, outer, k4 = {}, {}, {}
    tris, k4s = _cliques_and_triangles(n, N, rank)
    for x, y, z in tris:
        for (a, b), w in (((x, y), z), ((x, z), y), ((y, z), x)):
            e = key(a, b)
            opp[e] = opp.get(e, 0) + d[w] - opp_off
            outer[e] = outer.get(e, 0) + t[key(a, w)] + t[key(b, w)] - outer_off
    for q in k4s:
        for a, b in itertools.combinations(q, 2):
            k4[key(a, b)] = k4.get(key(a, b), 0) + 1
    c4, _ = _pivot_c4(n, N, rank, c4_off)
    rows = []
    for e in sorted(t):
        u, v = e
        te = t[e]
        n_pend = (s[v] - (d[u] - 1) - te) + (s[u] - (d[v] - 1) - te)
        n_pmid = (d[u] - 1) * (d[v] - 1) - te
        n_star = math.comb(d[u] - 1, 2) + math.comb(d[v] - 1, 2)
        n_tail = (tri[u] - te) + (tri[v] - te)
        n_att = te * (d[u] + d[v] - 4)
        n_chord = math.comb(te, 2)
        i9 = k4.get(e, 0)
        i8 = n_chord - i9
        i7 = outer.get(e, 0) - 4 * i9
        i6 = n_att - 4 * i8 - i7 - 4 * i9
        i5 = opp.get(e, 0) - i7 - 2 * i9
        i4 = n_tail - i7 - 2 * i9
        i3 = c4.get(e, 0) - i7 - 2 * i9
        i2 = n_star - i6 - i4 - 2 * i8 - i7 - 2 * i9
        i1 = n_pmid - i3 - i6 - 2 * i8 - i7 - 2 * i9
        i0 = n_pend - 2 * i3 - 2 * i5 - 2 * i4 - 3 * i7 - 4 * i9
        rows.append([i0, i1, i2, i3, i4, i5, i6, i7, i8, i9])
    return sorted(t), rows


def vertex_rows_by_kernel_rules(n, edges, rank):
    N = _graph(n, edges)
    d = [len(x) for x in N]
    key = lambda a, b: (min(a, b), max(a, b))
    t = {key(a, b): len(N[a] & N[b]) for a, b in edges}
    tri = [sum(t[key(x, w)] for w in N[x]) // 2 for x in range(n)]
    s = [sum(d[w] - 1 for w in N[x]) for x in range(n)]
    d2 = [0] * n
    k4 = [0] * n
    tris, k4s = _cliques_and_triangles(n, N, rank)
    for x, y, z in tris:   # each corner: t of the opposite edge - 1
        d2[x] += t[key(y, z)] - 1
        d2[y] += t[key(x, z)] - 1
        d2[z] += t[key(x, y)] - 1
    for q in k4s:
        for x in q:
            k4[x] += 1
    _, c4 = _pivot_c4(n, N, rank)
    rows = []
    for v in range(n):
        dv = d[v]
        pe = sum(s[u] - (dv - 1) for u in N[v]) - 2 * tri[v]
        pm = sum((dv - 1) * (d[u] - 1) - t[key(v, u)] for u in N[v])
        sl = sum(math.comb(d[u] - 1, 2) for u in N[v])
        sc = math.comb(dv, 3)
        tl = sum(tri[u] - t[key(v, u)] for u in N[v])
        to = sum(t[key(v, u)] * (d[u] - 2) for u in N[v])
        ta = tri[v] * (dv - 2)
        d3 = sum(math.comb(t[key(v, u)], 2) for u in N[v])
        o14 = k4[v]
        o13 = d3 - 3 * o14
        o12 = d2[v] - 3 * o14
        o11 = ta - 2 * o13 - 3 * o14
        o10 = to - 2 * o12 - 2 * o13 - 6 * o14
        o9 = tl - 2 * o12 - 3 * o14
        o8 = c4[v] - o12 - o13 - 3 * o14
        o7 = sc - o11 - o13 - o14
        o6 = sl - o9 - o10 - 2 * o12 - o13 - 3 * o14
        o5 = pm - 2 * o8 - o10 - 2 * o11 - 2 * o12 - 4 * o13 - 6 * o14
        o4 = pe - 2 * o8 - 2 * o9 - o10 - 4 * o12 - 2 * o13 - 6 * o14
        rows.append([o4, o5, o6, o7, o8, o9, o10, o11, o12, o13, o14])
    return rows


def test_vertex_kernel_rules_match_the_census():
    rng = np.random.default_rng(505)
    seen = np.zeros(11, bool)
    for trial in range(60):
        n = int(rng.integers(4, 17))
        edges = random_graph(rng, n, float(rng.uniform(0.05, 0.95)))
        rank = [int(x) for x in rng.permutation(n)]
        got = vertex_rows_by_kernel_rules(n, edges, rank)
        assert got == brute.vertex_orbit_census(n, edges), trial
        seen |= np.asarray(got).max(axis=0) > 0
    assert seen.all()


def test_edge_kernel_rules_match_the_census():
    rng = np.random.default_rng(404)
    seen = np.zeros(10, bool)
    for trial in range(60):
        n = int(rng.integers(4, 17))
        edges = random_graph(rng, n, float(rng.uniform(0.05, 0.95)))
        rank = [int(x) for x in rng.permutation(n)]
        got = edge_rows_by_kernel_rules(n, edges, rank)
        assert got == brute.edge_orbit_census(n, edges), trial
        if got[1]:
            seen |= np.asarray(got[1]).max(axis=0) > 0
    assert seen.all()


def test_pivot_cycle_credit_is_the_cycles_through_each_vertex_and_edge():
    """The 4-cycle walk from the highest vertex credits every non-induced
    4-cycle once to each of its four vertices and four edges, whatever the
    vertex order."""
    rng = np.random.default_rng(8)
    for trial in range(40):
        n = int(rng.integers(4, 13))
        edges = random_graph(rng, n, float(rng.uniform(0.1, 0.9)))
        N = _graph(n, edges)
        cyc_v = [0] * n
        cyc_e = {}
        for a, b, c, dd in itertools.permutations(range(n), 4):
            # each 4-cycle appears 8 times as a closed walk a-b-c-d-a
            if b in N[a] and c in N[b] and dd in N[c] and a in N[dd]:
                for x in (a, b, c, dd):
                    cyc_v[x] += 1
                for x, y in ((a, b), (b, c), (c, dd), (dd, a)):
                    e = (min(x, y), max(x, y))
                    cyc_e[e] = cyc_e.get(e, 0) + 1
        rank = [int(x) for x in rng.permutation(n)]
        edge, vert = _pivot_c4(n, N, rank)
        assert vert == [x // 8 for x in cyc_v], trial
        assert {e: x for e, x in edge.items() if x} == {e: x // 8 for e, x in cyc_e.items()}, trial


def test_planted_mistakes_in_the_edge_rules_fail():
    """Each credit constant off by one makes the census check fail on the
    same random graphs (so the test above can tell them apart)."""
    rng = np.random.default_rng(404)
    graphs = []
    for _ in range(60):
        n = int(rng.integers(4, 17))
        graphs.append((n, random_graph(rng, n, float(rng.uniform(0.05, 0.95))), [int(x) for x in rng.permutation(n)]))
    for bad in ({"opp_off": 1}, {"outer_off": 1}, {"outer_off": 3}, {"c4_off": 0}):
        assert any(edge_rows_by_kernel_rules(n, e, r, **bad) != brute.edge_orbit_census(n, e) for n, e, r in graphs), bad
