"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here runs CUDA.  Each test checks the oracle against something other
than itself: hand-derived counts of named graphs, a brute-force census of
every 4-subset, containment numbers enumerated from first principles, and the
identities that Lemma 1 / Lemma 2 (Sec. 4.2, 4.3) guarantee for the dynamic
update.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import gen
from gc_testutil import (bfs_region, csr_from_edges, edges_from_csr, load_closed_forms,
                         random_graph, rows_of)

CLOSED = load_closed_forms()


# ---------------------------------------------------------------- static --

@pytest.mark.parametrize("name,n,edges,expect", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_form_graphs(name, n, edges, expect, oracle_lib):
    rp, col = csr_from_edges(n, edges)
    assert brute.graphlet_counts(n, edges) == expect
    assert oracle.static_counts(rp, col, "literal") == expect
    assert oracle.static_counts(rp, col, "oriented") == expect


def test_complete_graph_family(oracle_lib):
    for n in range(4, 11):
        rp, col = csr_from_edges(n, itertools.combinations(range(n), 2))
        assert oracle.static_counts(rp, col, "oriented") == [0, 0, 0, 0, 0, math.comb(n, 4)]
        assert oracle.static_counts(rp, col, "literal") == [0, 0, 0, 0, 0, math.comb(n, 4)]


def test_bipartite_and_cycle_families(oracle_lib):
    for a in range(1, 6):
        for b in range(1, 7):
            n = a + b
            rp, col = csr_from_edges(n, [(i, a + j) for i in range(a) for j in range(b)])
            exp = [0, a * math.comb(b, 3) + b * math.comb(a, 3), math.comb(a, 2) * math.comb(b, 2), 0, 0, 0]
            assert oracle.static_counts(rp, col, "oriented") == exp
    for n in range(5, 12):
        rp, col = csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
        assert oracle.static_counts(rp, col, "oriented") == [n, 0, 0, 0, 0, 0]
        rp, col = csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
        assert oracle.static_counts(rp, col, "literal") == [n - 3, 0, 0, 0, 0, 0]


def test_census_covers_every_subset():
    rng = np.random.default_rng(7)
    for _ in range(40):
        n = int(rng.integers(4, 13))
        h = brute.census(n, random_graph(rng, n, rng.random()))
        assert sum(h.values()) == math.comb(n, 4)


def _classify_edges(edge_subset):
    deg = {}
    for a, b in edge_subset:
        deg[a] = deg.get(a, 0) + 1
        deg[b] = deg.get(b, 0) + 1
    return len(edge_subset), tuple(sorted(deg.get(v, 0) for v in range(4)))


# representative of each connected graphlet on vertices 0..3
_SHAPES = {
    "g1": [(0, 1), (1, 2), (2, 3)],
    "g2": [(0, 1), (0, 2), (0, 3)],
    "g3": [(0, 1), (1, 2), (2, 3), (3, 0)],
    "g4": [(0, 1), (1, 2), (2, 0), (2, 3)],
    "g5": [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)],
    "g6": [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)],
}
_PATTERN_SIG = {  # (edges, sorted degrees) of each non-induced pattern
    "P": (3, (1, 1, 2, 2)), "S": (3, (1, 1, 1, 3)), "TT": (4, (1, 2, 2, 3)),
    "D": (5, (2, 2, 3, 3)), "K": (6, (3, 3, 3, 3)), "Q": (4, (2, 2, 2, 2)),
}


def _containment():
    """copies[pattern][graphlet]: edge subsets of the graphlet shaped like the pattern."""
    out = {p: {} for p in _PATTERN_SIG}
    for g, edges in _SHAPES.items():
        for p, sig in _PATTERN_SIG.items():
            c = 0
            for r in range(len(edges) + 1):
                for sub in itertools.combinations(edges, r):
                    if _classify_edges(sub) == sig:
                        c += 1
            out[p][g] = c
    return out


def test_containment_matrix_by_enumeration():
    c = _containment()
    # spot values quoted in the oracle's header
    assert [c["D"]["g6"], c["Q"]["g6"], c["TT"]["g6"], c["S"]["g6"], c["P"]["g6"]] == [6, 3, 12, 4, 12]
    assert [c["Q"]["g5"], c["TT"]["g5"], c["S"]["g5"], c["P"]["g5"]] == [1, 4, 2, 6]
    assert c["P"]["g3"] == 4 and c["S"]["g4"] == 1 and c["P"]["g4"] == 2


def test_each_sum_matches_brute_force(oracle_lib):
    """Every non-induced sum equals the census pushed through the enumerated
    containment matrix, so a dropped or mis-signed term in any single sum fails."""
    cont = _containment()
    rng = np.random.default_rng(11)
    for trial in range(150):
        n = int(rng.integers(4, 15))
        edges = random_graph(rng, n, float(rng.random()))
        h = brute.census(n, edges)
        expect = [sum(cont[p][g] * h[g] for g in _SHAPES) for p in ("P", "S", "TT", "D", "K", "Q")]
        rp, col = csr_from_edges(n, edges)
        lit = oracle.sums_literal(rp, col, with_ic4=True)
        assert lit[:6] == expect, (trial, n)
        assert lit[6] == h["g3"]  # PGD's per-edge induced 4-cycle rule
        assert oracle.sums_oriented(rp, col) == expect, (trial, n)
        assert oracle.counts_from_sums(expect) == [h[g] for g in brute.CONNECTED]


def test_planted_hubs_and_cliques(oracle_lib):
    """Dense cores plus a hub: exercises large t_uv and high-degree pivots."""
    rng = np.random.default_rng(3)
    for trial in range(30):
        n = 30
        edges = set(map(tuple, random_graph(rng, n, 0.08)))
        core = rng.choice(n, size=7, replace=False)
        edges |= {(min(a, b), max(a, b)) for a in core for b in core if a != b}
        hub = int(rng.integers(0, n))
        edges |= {(min(hub, v), max(hub, v)) for v in range(n) if v != hub and rng.random() < 0.7}
        edges = sorted(edges)
        rp, col = csr_from_edges(n, edges)
        bf = brute.graphlet_counts(n, edges)
        assert oracle.static_counts(rp, col, "literal") == bf
        assert oracle.static_counts(rp, col, "oriented") == bf


def test_variants_agree_on_workload_graphs(oracle_lib):
    for name in ("c1", "c2"):
        n, keys = gen.workload_graph(name)
        rp, col = gen.csr_from_keys(n, keys)
        assert oracle.sums_literal(rp, col) == oracle.sums_oriented(rp, col)


def test_relabel_invariance(oracle_lib):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    base = oracle.static_counts(rp, col)
    perm = np.random.default_rng(5).permutation(n)
    edges = [(int(perm[a]), int(perm[b])) for a, b in edges_from_csr(rp, col)]
    rp2, col2 = csr_from_edges(n, edges)
    assert oracle.static_counts(rp2, col2) == base


# --------------------------------------------------------------- dynamic --

def _random_dirty_batch(rng, n, edges, k_ins, k_del):
    """Pairs with repeats, reversed orientation, cancellations and no-ops."""
    es = list(edges)
    ins = [tuple(rng.choice(n, 2, replace=False)) for _ in range(k_ins)]
    dels = [es[i] for i in rng.choice(len(es), min(k_del, len(es)), replace=False)] if es else []
    dels += [tuple(rng.choice(n, 2, replace=False)) for _ in range(k_del // 3)]
    if ins and rng.random() < 0.5:
        dels.append(ins[0][::-1])          # cancelled pair
    if dels and rng.random() < 0.5:
        ins.append(dels[0])                # cancelled pair
    if ins:
        ins.append(ins[-1][::-1])          # repeat, reversed
    ins = np.array(ins, dtype=np.int32).reshape(-1, 2)
    dels = np.array(dels, dtype=np.int32).reshape(-1, 2)
    return ins, dels


def test_lemma2_on_random_graphs(oracle_lib):
    """Algorithm 2: F + C_a - C_b equals the census of G \\ D u A (Lemma 2)."""
    rng = np.random.default_rng(21)
    for trial in range(120):
        n = int(rng.integers(5, 16))
        edges = random_graph(rng, n, float(rng.uniform(0.1, 0.7)))
        rp, col = csr_from_edges(n, edges)
        F0 = brute.graphlet_counts(n, edges)
        ins, dels = _random_dirty_batch(rng, n, edges, int(rng.integers(0, 5)), int(rng.integers(0, 5)))
        for variant in ("literal", "oriented"):
            r = oracle.fdgc_step(rp, col, ins, dels, F0, 3, variant)
            after = edges_from_csr(r["row_ptr"], r["col"])
            assert r["F"] == brute.graphlet_counts(n, after), (trial, variant)
        # the committed graph is G \ D u A after normalisation
        A, D, _ = oracle.normalize(rp, col, ins, dels)
        eset = {(a << 32) | b for a, b in edges}
        expect = (eset - set(map(int, D))) | set(map(int, A))
        assert {(a << 32) | b for a, b in after} == expect


def test_lemma2_workload_c1(oracle_lib):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.random_batch(n, keys, 200, 200, 1, ins_weighting="uniform")
    F0 = oracle.static_counts(rp, col, "literal")
    r = oracle.fdgc_step(rp, col, ins, dels, F0, 3, "literal")
    assert (r["n_ins"], r["n_del"]) == (200, 200)
    assert r["F"] == oracle.static_counts(r["row_ptr"], r["col"], "literal")
    assert [a - b for a, b in zip(r["Ca"], r["Cb"])] == [x - y for x, y in zip(r["F"], F0)]


def test_lemma2_workload_c2_stream(oracle_lib):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    g = oracle.OracleGraph(rp, col)
    for ins, dels in gen.batch_stream(n, keys, [1000, 10000, 1000], 0.5, 2):
        g.apply(ins, dels)
        assert g.F == oracle.static_counts(g.row_ptr, g.col)
    # insert-only (IGC) stream
    g = oracle.OracleGraph(rp, col)
    for ins, dels in gen.batch_stream(n, keys, [1000, 10000], 1.0, 2):
        assert len(dels) == 0
        g.apply(ins, dels)
        assert g.F == oracle.static_counts(g.row_ptr, g.col)


def test_radius_two_suffices_and_one_does_not(oracle_lib):
    """Any 4-subset holding a changed pair lies within 2 hops of its
    endpoints, so k = 2 gives the same delta as the paper's k = 3; k = 1
    misses subsets and must fail somewhere."""
    rng = np.random.default_rng(31)
    k1_wrong = 0
    for trial in range(150):
        n = int(rng.integers(6, 16))
        edges = random_graph(rng, n, float(rng.uniform(0.1, 0.5)))
        rp, col = csr_from_edges(n, edges)
        F0 = oracle.static_counts(rp, col)
        ins, dels = _random_dirty_batch(rng, n, edges, 2, 2)
        r3 = oracle.fdgc_step(rp, col, ins, dels, F0, 3)
        r2 = oracle.fdgc_step(rp, col, ins, dels, F0, 2)
        r1 = oracle.fdgc_step(rp, col, ins, dels, F0, 1)
        assert r2["F"] == r3["F"]
        k1_wrong += r1["F"] != r3["F"]
    assert k1_wrong > 0


def test_region_is_the_same_in_G_and_G_union_A(oracle_lib):
    """The walk starts from every endpoint, so an inserted edge joins two
    vertices already at depth 0 and can never shorten a distance: the region
    taken in G (Algorithm 2 as printed) equals the region taken in G u A."""
    rng = np.random.default_rng(41)
    for trial in range(60):
        n = int(rng.integers(6, 30))
        edges = random_graph(rng, n, float(rng.uniform(0.05, 0.3)))
        rp, col = csr_from_edges(n, edges)
        ins, dels = _random_dirty_batch(rng, n, edges, 3, 3)
        r = oracle.fdgc_step(rp, col, ins, dels, [0] * 6, 3, want_region=True)
        A, D, _ = oracle.normalize(rp, col, ins, dels)
        src = [int(k >> 32) for k in list(A) + list(D)] + [int(k & 0xFFFFFFFF) for k in list(A) + list(D)]
        expect = bfs_region(n, rows_of(rp, col), src, 3)
        assert list(map(int, r["region"])) == expect


def test_igc_is_fdgc_without_deletions(oracle_lib):
    """Algorithm 1 built literally (G <- G + B first, W from the updated
    graph, G_b = G_a \\ B) gives the same C_a and C_b as Algorithm 2 with
    D empty."""
    rng = np.random.default_rng(51)
    for trial in range(60):
        n = int(rng.integers(6, 20))
        edges = random_graph(rng, n, float(rng.uniform(0.1, 0.4)))
        rp, col = csr_from_edges(n, edges)
        eset = set(edges)
        cand = [(a, b) for a in range(n) for b in range(a + 1, n) if (a, b) not in eset]
        if not cand:
            continue
        pick = rng.choice(len(cand), min(len(cand), int(rng.integers(1, 5))), replace=False)
        B = [cand[i] for i in pick]
        new_edges = sorted(eset | set(B))
        rp1, col1 = csr_from_edges(n, new_edges)
        W = bfs_region(n, rows_of(rp1, col1), [x for e in B for x in e], 3)
        idx = {v: i for i, v in enumerate(W)}
        ga = [(idx[a], idx[b]) for a, b in new_edges if a in idx and b in idx]
        gb = [e for e in ga if (W[e[0]], W[e[1]]) not in set(B)]
        Ca = oracle.static_counts(*csr_from_edges(len(W), ga))
        Cb = oracle.static_counts(*csr_from_edges(len(W), gb))
        r = oracle.fdgc_step(rp, col, np.array(B, dtype=np.int32), np.zeros((0, 2), np.int32), [0] * 6, 3)
        assert (r["Ca"], r["Cb"]) == (Ca, Cb)


def test_batch_then_inverse_restores_counts(oracle_lib):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    g = oracle.OracleGraph(rp, col)
    F0 = list(g.F)
    ins, dels = gen.random_batch(n, keys, 700, 300, 9)
    g.apply(ins, dels)
    assert g.F != F0
    g.apply(dels, ins)
    assert g.F == F0
    assert np.array_equal(g.row_ptr, rp.astype(np.int64)) and np.array_equal(g.col, col)


def test_split_batch_gives_same_counts(oracle_lib):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.random_batch(n, keys, 200, 200, 1, ins_weighting="uniform")
    whole = oracle.OracleGraph(rp, col)
    whole.apply(ins, dels)
    parts = oracle.OracleGraph(rp, col)
    parts.apply(ins[:77], dels[:150])
    parts.apply(ins[77:], dels[150:])
    assert whole.F == parts.F


def test_normalisation_rules(oracle_lib):
    # path 0-1-2-3 plus edge 0-2
    rp, col = csr_from_edges(5, [(0, 1), (1, 2), (2, 3), (0, 2)])
    ins = np.array([[3, 4], [4, 3], [1, 3], [0, 1], [2, 4]], dtype=np.int32)
    dels = np.array([[2, 1], [1, 2], [0, 4], [3, 1]], dtype=np.int32)
    A, D, st = oracle.normalize(rp, col, ins, dels)
    # (3,4) repeated -> once; (1,3) also deleted -> cancelled; (0,1) exists -> no-op
    assert sorted(int(k) for k in A) == [(2 << 32) | 4, (3 << 32) | 4]
    # (1,2) repeated -> once; (0,4) missing -> no-op; (1,3) cancelled
    assert [int(k) for k in D] == [(1 << 32) | 2]
    assert st == [5, 4, 1, 1, 1, 1, 1, 0]
    with pytest.raises(ValueError):
        oracle.normalize(rp, col, np.array([[2, 2]], np.int32), np.zeros((0, 2), np.int32))
    with pytest.raises(ValueError):
        oracle.normalize(rp, col, np.zeros((0, 2), np.int32), np.array([[0, 5]], np.int32))


def test_empty_and_all_noop_batches(oracle_lib):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    e = np.zeros((0, 2), np.int32)
    r = oracle.fdgc_step(rp, col, e, e, F0)
    assert r["F"] == F0 and r["region_vertices"] == 0 and r["Ca"] == [0] * 6
    existing = np.array(edges_from_csr(rp, col)[:10], dtype=np.int32)
    r = oracle.fdgc_step(rp, col, existing, np.array([[0, 1999]] if 1999 not in col[rp[0]:rp[1]] else [], np.int32).reshape(-1, 2), F0)
    assert r["F"] == F0 and r["region_vertices"] == 0 and r["noops"] >= 10


def test_stored_workload_values(oracle_lib):
    """``golden/workloads.json`` (written by ``golden/make_golden.py`` from the
    oracle alone) still matches a fresh oracle run, and is self-consistent
    with Lemma 2."""
    import json
    import os

    from gc_testutil import GOLDEN_DIR

    with open(os.path.join(GOLDEN_DIR, "workloads.json")) as f:
        gold = json.load(f)
    c1 = gold["c1"]
    assert [a - b for a, b in zip(c1["Ca"], c1["Cb"])] == [x - y for x, y in zip(c1["after"], c1["static"])]
    assert oracle.counts_from_sums(c1["sums_a"]) == c1["Ca"]
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    assert oracle.static_counts(rp, col) == c1["static"]
    ins, dels = gen.random_batch(n, keys, 200, 200, 1, ins_weighting="uniform")
    r = oracle.fdgc_step(rp, col, ins, dels, c1["static"], 3)
    assert r["F"] == c1["after"] and r["Ca"] == c1["Ca"] and r["Cb"] == c1["Cb"]
    assert oracle.static_counts(r["row_ptr"], r["col"], "literal") == c1["after"]


# ------------------------------------------------------- 3-vertex graphlets --

def test_counts3_closed_forms(oracle_lib):
    """[induced 2-paths, triangles]: K_n has C(n,3) triangles and no open
    path; the star K_1,s has C(s,2) open paths; P_n has n - 2; C_n (n >= 4)
    has n; K_a,b has a C(b,2) + b C(a,2)."""
    def kn(n):
        return n, [(a, b) for a in range(n) for b in range(a + 1, n)]

    cases = []
    for n in (3, 4, 7):
        cases.append((kn(n), [0, math.comb(n, 3)]))
    for s in (3, 6):
        cases.append(((s + 1, [(0, i) for i in range(1, s + 1)]), [math.comb(s, 2), 0]))
    for n in (3, 6):
        cases.append(((n, [(i, i + 1) for i in range(n - 1)]), [n - 2, 0]))
    for n in (4, 9):
        cases.append(((n, [(i, (i + 1) % n) for i in range(n)]), [n, 0]))
    for a, b in ((2, 3), (3, 4)):
        edges = [(i, a + j) for i in range(a) for j in range(b)]
        cases.append(((a + b, edges), [a * math.comb(b, 2) + b * math.comb(a, 2), 0]))
    for (n, edges), expect in cases:
        rp, col = csr_from_edges(n, edges)
        assert oracle.static_counts3(rp, col) == expect
        assert brute.graphlet3_counts(n, edges) == expect


def test_counts3_match_census_on_random_graphs(oracle_lib):
    rng = np.random.default_rng(33)
    for _ in range(80):
        n = int(rng.integers(3, 20))
        edges = random_graph(rng, n, float(rng.uniform(0.1, 0.8)))
        rp, col = csr_from_edges(n, edges)
        h = brute.census3(n, edges)
        assert sum(h.values()) == math.comb(n, 3)
        assert oracle.static_counts3(rp, col) == [h["path"], h["triangle"]]


def test_counts3_triangles_agree_with_the_four_vertex_sums(oracle_lib):
    """Triangles from the 3-vertex count equal a third of the sum of t_e that
    the 4-vertex sums use: TT = 1/2 sum t_e (d_u + d_v - 4) on a graph whose
    every edge has d_u + d_v = 6 gives TT = sum t_e = 3 triangles (the
    3-regular graphs K_4 and the prism)."""
    k4 = (4, [(a, b) for a in range(4) for b in range(a + 1, 4)])
    prism = (6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (0, 3), (1, 4), (2, 5)])
    for n, edges in (k4, prism):
        rp, col = csr_from_edges(n, edges)
        tri = oracle.static_counts3(rp, col)[1]
        TT = oracle.sums_literal(rp, col)[2]
        assert TT == 3 * tri


def test_all_eleven_types_match_the_census(oracle_lib):
    """The disconnected types from closed forms against the census of every
    4-subset (Problem 1's six graphlets plus the five disconnected graphs)."""
    rng = np.random.default_rng(4411)
    order = ["g1", "g2", "g3", "g4", "g5", "g6", "triangle+isolated", "wedge+isolated", "two-edges", "edge", "empty"]
    for trial in range(40):
        n = int(rng.integers(4, 22))
        p = float(rng.uniform(0.0, 0.9))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        rp, col = csr_from_edges(n, edges)
        h = brute.census(n, edges)
        assert oracle.counts_all(rp, col) == [h[k] for k in order], trial
        assert sum(oracle.counts_all(rp, col)) == math.comb(n, 4)


def test_vertex_counts_match_the_census(oracle_lib):
    """Per-vertex graphlet counts against the census of every 4-subset
    credited to its four vertices; their sum over vertices is four times
    the global counts."""
    rng = np.random.default_rng(909)
    for trial in range(50):
        n = int(rng.integers(4, 20))
        p = float(rng.uniform(0.05, 0.95))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        rp, col = csr_from_edges(n, edges)
        got = oracle.vertex_counts(rp, col)
        assert got == brute.vertex_census(n, edges), trial
        tot = [sum(r[k] for r in got) for k in range(6)]
        assert tot == [4 * x for x in oracle.static_counts(rp, col)]


def test_vertex_counts_of_named_graphs(oracle_lib):
    # K4: one 4-clique through each vertex; C4: one 4-cycle; the star K_{1,3}:
    # one 3-star through each vertex; P4: one 3-path
    for n, edges, k in ((4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], 5),
                        (4, [(0, 1), (1, 2), (2, 3), (3, 0)], 2),
                        (4, [(0, 1), (0, 2), (0, 3)], 1),
                        (4, [(0, 1), (1, 2), (2, 3)], 0)):
        rp, col = csr_from_edges(n, edges)
        want = [[1 if j == k else 0 for j in range(6)] for _ in range(n)]
        assert oracle.vertex_counts(rp, col) == want


def test_vertex_orbits_match_the_census(oracle_lib):
    """Orbit counts per vertex (orbits 4..14) against the census of every
    4-subset, each vertex credited with its orbit in the induced graph."""
    rng = np.random.default_rng(1414)
    seen = np.zeros(11, bool)
    for trial in range(50):
        n = int(rng.integers(4, 20))
        p = float(rng.uniform(0.05, 0.95))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        rp, col = csr_from_edges(n, edges)
        got = oracle.vertex_orbits(rp, col)
        assert got == brute.vertex_orbit_census(n, edges), trial
        seen |= np.asarray(got).max(axis=0) > 0
    assert seen.all()   # every orbit occurs, so every term of the inversion is exercised


def _role_counts_by_enumeration():
    """For each connected 4-vertex graph g and each vertex orbit o in it,
    the number of non-induced copies of each subgraph H (3-path, 3-star,
    4-cycle, tailed triangle, diamond, 4-clique) that hold that vertex in
    each role, found by trying every edge subset of g: the matrix the
    per-vertex orbit inversion uses."""
    graphs = {  # one representative of each type on vertices 0..3
        "g1": [(0, 1), (1, 2), (2, 3)],
        "g2": [(0, 1), (0, 2), (0, 3)],
        "g3": [(0, 1), (1, 2), (2, 3), (3, 0)],
        "g4": [(0, 1), (1, 2), (2, 0), (2, 3)],
        "g5": [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)],
        "g6": [(a, b) for a in range(4) for b in range(a + 1, 4)],
    }

    def role(edges, v):
        deg = [0] * 4
        for a, b in edges:
            deg[a] += 1
            deg[b] += 1
        cls = brute._CLASSES.get((len(edges), tuple(sorted(deg))))
        if cls not in brute.CONNECTED:
            return None
        return brute._orbit(cls, deg, v)   # the role of v in the copy = its orbit in that graph

    table = {}
    for g, edges in graphs.items():
        for v in range(4):
            deg = [0] * 4
            for a, b in edges:
                deg[a] += 1
                deg[b] += 1
            o = brute._orbit(g, deg, v)
            counts = {}
            for r in range(1, len(edges) + 1):
                for sub in itertools.combinations(edges, r):
                    # a copy spans all four vertices
                    if len({x for e in sub for x in e}) != 4:
                        continue
                    rr = role(list(sub), v)
                    if rr is not None:
                        counts[rr] = counts.get(rr, 0) + 1
            table[o] = counts
    return table


def test_role_containment_by_enumeration():
    """The coefficients of the per-vertex orbit inversion, enumerated from
    the edge subsets of each graphlet (orbit -> {role: copies})."""
    t = _role_counts_by_enumeration()
    assert t[14] == {4: 6, 5: 6, 6: 3, 7: 1, 8: 3, 9: 3, 10: 6, 11: 3, 12: 3, 13: 3, 14: 1}
    assert t[13] == {4: 2, 5: 4, 6: 1, 7: 1, 8: 1, 10: 2, 11: 2, 13: 1}
    assert t[12] == {4: 4, 5: 2, 6: 2, 8: 1, 9: 2, 10: 2, 12: 1}
    assert t[11] == {5: 2, 7: 1, 11: 1}
    assert t[10] == {4: 1, 5: 1, 6: 1, 10: 1}
    assert t[9] == {4: 2, 6: 1, 9: 1}
    assert t[8] == {4: 2, 5: 2, 8: 1}
    assert t[7] == {7: 1} and t[6] == {6: 1} and t[5] == {5: 1} and t[4] == {4: 1}


# ------------------------------------------------------- per-edge orbits --

def test_edge_orbits_match_the_census(oracle_lib):
    """Edge orbit counts (10 columns) against the census of every 4-subset,
    each edge of the induced graph credited with its orbit there."""
    rng = np.random.default_rng(2020)
    seen = np.zeros(10, bool)
    for trial in range(60):
        n = int(rng.integers(4, 18))
        p = float(rng.uniform(0.05, 0.95))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        rp, col = csr_from_edges(n, edges)
        got = oracle.edge_orbits(rp, col)
        assert got == brute.edge_orbit_census(n, edges), trial
        if got[1]:
            seen |= np.asarray(got[1]).max(axis=0) > 0
    assert seen.all()   # every edge orbit occurs, so every term of the inversion is exercised


def test_edge_orbits_of_named_graphs(oracle_lib):
    c2 = lambda x: x * (x - 1) // 2
    for n in range(4, 9):   # K_n: every edge lies in C(n-2, 2) 4-cliques
        edges = list(itertools.combinations(range(n), 2))
        rp, col = csr_from_edges(n, edges)
        assert oracle.edge_orbits(rp, col)[1] == [[0] * 9 + [c2(n - 2)]] * len(edges)
    for n in range(5, 10):  # C_n: each edge ends two 3-paths and is the middle of one
        edges = [(i, (i + 1) % n) for i in range(n)]
        rp, col = csr_from_edges(n, edges)
        assert oracle.edge_orbits(rp, col)[1] == [[2, 1] + [0] * 8] * n
    for a in range(1, 5):   # K_{a,b}: 3-stars at either end and (a-1)(b-1) 4-cycles
        for b in range(1, 6):
            edges = [(i, a + j) for i in range(a) for j in range(b)]
            rp, col = csr_from_edges(a + b, edges)
            want = [0, 0, c2(b - 1) + c2(a - 1), (a - 1) * (b - 1), 0, 0, 0, 0, 0, 0]
            assert oracle.edge_orbits(rp, col)[1] == [want] * len(edges), (a, b)


def test_edge_orbits_sum_to_the_global_counts(oracle_lib):
    """Summed over edges, each orbit gives its graphlet count times the
    number of its edges in that orbit (3-path 2 + 1, 3-star 3, 4-cycle 4,
    tailed triangle 1 + 1 + 2, diamond 4 + 1, 4-clique 6); the global counts
    come from the C oracle."""
    rng = np.random.default_rng(3)
    for n, p in ((120, 0.08), (60, 0.4)):
        edges = random_graph(rng, n, p)
        rp, col = csr_from_edges(n, edges)
        rows = np.asarray(oracle.edge_orbits(rp, col)[1], dtype=np.int64)
        tot = rows.sum(axis=0).tolist()
        g1, g2, g3, g4, g5, g6 = oracle.static_counts(rp, col)
        assert tot == [2 * g1, g1, 3 * g2, 4 * g3, g4, g4, 2 * g4, 4 * g5, g5, 6 * g6]


def _edge_role_counts_by_enumeration():
    """For each connected 4-vertex graph g and each edge orbit in it, the
    number of non-induced copies of each connected subgraph holding that
    edge in each edge role, found by trying every edge subset of g: the
    matrix the per-edge orbit inversion uses."""
    graphs = {
        "g1": [(0, 1), (1, 2), (2, 3)],
        "g2": [(0, 1), (0, 2), (0, 3)],
        "g3": [(0, 1), (1, 2), (2, 3), (3, 0)],
        "g4": [(0, 1), (1, 2), (2, 0), (2, 3)],
        "g5": [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)],
        "g6": [(a, b) for a in range(4) for b in range(a + 1, 4)],
    }

    def degs(edges):
        d = [0] * 4
        for a, b in edges:
            d[a] += 1
            d[b] += 1
        return d

    table = {}
    for g, edges in graphs.items():
        for e in edges:
            o = brute._edge_orbit(g, degs(edges), *e)
            counts = {}
            for r in range(1, len(edges) + 1):
                for sub in itertools.combinations(edges, r):
                    if e not in sub or len({x for f in sub for x in f}) != 4:
                        continue
                    d = degs(sub)
                    cls = brute._CLASSES.get((len(sub), tuple(sorted(d))))
                    if cls in brute.CONNECTED:
                        rr = brute._edge_orbit(cls, d, *e)
                        counts[rr] = counts.get(rr, 0) + 1
            assert table.setdefault(o, counts) == counts   # one answer per orbit
    return table


def test_edge_role_containment_by_enumeration():
    """The coefficients of the per-edge orbit inversion (orbit -> {role:
    copies}), enumerated from the edge subsets of each graphlet."""
    t = _edge_role_counts_by_enumeration()
    assert t[9] == {0: 4, 1: 2, 2: 2, 3: 2, 4: 2, 5: 2, 6: 4, 7: 4, 8: 1, 9: 1}
    assert t[8] == {1: 2, 2: 2, 6: 4, 8: 1}
    assert t[7] == {0: 3, 1: 1, 2: 1, 3: 1, 4: 1, 5: 1, 6: 1, 7: 1}
    assert t[6] == {1: 1, 2: 1, 6: 1}
    assert t[5] == {0: 2, 5: 1}
    assert t[4] == {0: 2, 2: 1, 4: 1}
    assert t[3] == {0: 2, 1: 1, 3: 1}
    assert t[2] == {2: 1} and t[1] == {1: 1} and t[0] == {0: 1}
