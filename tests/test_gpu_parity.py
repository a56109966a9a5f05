"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

Counts are integers and must match bit-exactly (uint64).  Expected values come
from the oracle, run here on the same seeded inputs, or from the stored
oracle results in golden/.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import gen
from gc_testutil import GOLDEN_DIR, csr_from_edges, edges_from_csr, load_closed_forms, random_graph

pytestmark = pytest.mark.gpu

CLOSED = load_closed_forms()


@pytest.fixture(scope="module")
def gcb():
    from paper_2308_14493_gb300 import gc as binding

    binding.load()
    return binding


def open_graph(gcb, n, rp, col, **kw):
    return gcb.Graph(n, rp, col, **kw)


def mod64(xs):
    return [int(x) & 0xFFFFFFFFFFFFFFFF for x in xs]


def same_graph(g, rp, col):
    grp, gcol = g.export_csr()
    return np.array_equal(grp.astype(np.int64), np.asarray(rp, np.int64)) and np.array_equal(gcol, np.asarray(col))


# ------------------------------------------------------------------ static --

@pytest.mark.parametrize("name,n,edges,expect", CLOSED, ids=[c[0] for c in CLOSED])
def test_static_named_graphs(gcb, name, n, edges, expect):
    rp, col = csr_from_edges(n, edges)
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts() == expect
        assert g.count_static() == expect


def test_static_random_small_graphs(gcb):
    rng = np.random.default_rng(101)
    for trial in range(60):
        n = int(rng.integers(1, 40))
        edges = random_graph(rng, n, float(rng.random()))
        rp, col = csr_from_edges(n, edges)
        with open_graph(gcb, n, rp, col) as g:
            expect = brute.graphlet_counts(n, edges) if n <= 20 else oracle.static_counts(rp, col, "literal")
            assert g.counts() == expect, (trial, n)


def test_static_planted_hub_and_clique(gcb):
    """A 2,000-vertex graph with a 600-degree hub and a 40-clique: exercises
    long rows, many triangles per edge and heavy 4-cycle pivots."""
    rng = np.random.default_rng(5)
    n = 2000
    keys = set(int(k) for k in gen.er_graph(n, 8000, 9))
    hub = 17
    for v in rng.choice(n, 600, replace=False):
        if v != hub:
            keys.add((min(hub, v) << 32) | max(hub, v))
    core = rng.choice(n, 40, replace=False)
    for a in core:
        for b in core:
            if a < b:
                keys.add((int(a) << 32) | int(b))
    k = np.array(sorted(keys), dtype=np.uint64)
    rp, col = gen.csr_from_keys(n, k)
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts() == oracle.static_counts(rp, col, "literal")


def _bipartite_hub_graph():
    """A pivot with 90,000 wedges onto 300 endpoints: hub h (350 neighbours:
    300 'a' vertices and 50 leaves), each 'a' joined to the same 300 'b'
    vertices, plus a sparse background."""
    n = 3000
    keys = set(int(k) for k in gen.er_graph(n, 3000, 21))
    h, A, B, L = 0, range(1, 301), range(301, 601), range(601, 651)
    for a in A:
        keys.add((h << 32) | a)
        for b in B:
            keys.add((a << 32) | b)
    for x in L:
        keys.add((h << 32) | x)
    k = np.array(sorted(keys), dtype=np.uint64)
    return n, k


CHUNK_CASES = [
    ("c2", dict(chunk_threshold=64)),
    ("hub", dict(chunk_threshold=64)),
    ("wide_ids", dict(chunk_threshold=64)),
    ("wide_ids", dict(chunk_threshold=4096)),
]


def _chunk_graph(name):
    if name == "c2":
        return gen.workload_graph("c2")
    if name == "hub":
        return _bipartite_hub_graph()
    # 120,000 ids: the chunked kernel's id range spans three chunks
    return 120000, gen.chung_lu_graph(120000, 400000, 2.1, 3000.0, 22)


@pytest.mark.parametrize("name,opts", CHUNK_CASES, ids=[f"{c[0]}-{'-'.join(map(str, c[1].values()))}"
                                                        for c in CHUNK_CASES])
def test_chunked_four_cycle_tier(gcb, name, opts):
    """4-cycle pivots counted in shared memory over id-range chunks (three
    chunks on the 120,000-vertex graph), with the tier taking every pivot
    above the hash tiers; static counts and a batch equal the oracle."""
    n, keys = _chunk_graph(name)
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    ins, dels = gen.random_batch(n, keys, 300, 200, 23)
    r = oracle.fdgc_step(rp, col, ins, dels, F0)
    with open_graph(gcb, n, rp, col, **opts) as g:
        assert g.counts() == F0
        assert g.count_static() == F0
        assert g.apply(ins, dels) == r["F"]
        st = g.stats()
        assert mod64(st["sums_a"]) == mod64(r["sums_a"]) and mod64(st["sums_b"]) == mod64(r["sums_b"])


TUNINGS = {
    "tri_all_merge": dict(tri_warp_max=1, tri_small_max=1, tri_block_max=1),
    "tri_all_block": dict(tri_warp_max=1, tri_small_max=1, tri_block_max=512),
    "tri_all_small_block": dict(tri_warp_max=1, tri_small_max=128, tri_block_max=128),
    "tri_small_block": dict(tri_warp_max=8, tri_small_max=20, tri_block_max=40),
    "c4_warp_hash": dict(c4_reg_max=1, c4_warp_max=512, c4_block_max=512, c4_cta_max=512),
    "c4_block_hash": dict(c4_reg_max=1, c4_warp_max=1, c4_block_max=8192, c4_cta_max=8192),
    "c4_small_block_hash": dict(c4_reg_max=1, c4_warp_max=1, c4_block_max=2048, c4_cta_max=2048),
    "c4_cta_hash": dict(c4_reg_max=1, c4_warp_max=1, c4_block_max=1, c4_cta_max=32768),
    "c4_all_cluster": dict(c4_reg_max=1, c4_warp_max=1, c4_block_max=1, c4_cta_max=1, c4_chunk_min=0),
    "c4_all_chunk": dict(c4_reg_max=1, c4_warp_max=1, c4_block_max=1, c4_cta_max=1, c4_chunk_min=1),
    "c4_chunk_then_cluster": dict(c4_reg_max=1, c4_warp_max=1, c4_block_max=1, c4_cta_max=1, c4_chunk_min=1,
                                  c4_chunk_max=2000),
}


@pytest.mark.parametrize("tname", sorted(TUNINGS))
@pytest.mark.parametrize("gname", ["c2", "hub"])
def test_every_kernel_tier_alone(gcb, gname, tname):
    """Bin boundaries move work between kernels, never change counts: with
    each tier forced to take (almost) every root or pivot, the static count
    and a batch equal the oracle."""
    n, keys = _chunk_graph(gname)
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    ins, dels = gen.random_batch(n, keys, 250, 250, 31)
    r = oracle.fdgc_step(rp, col, ins, dels, F0)
    with open_graph(gcb, n, rp, col) as g:
        g.set_tuning(**TUNINGS[tname])
        assert g.count_static() == F0
        assert g.apply(ins, dels) == r["F"]
        assert mod64(g.stats()["Ca"]) == mod64(r["Ca"])


def test_cluster_counters_with_many_one_graph_wedges(gcb):
    """The heavy-pivot kernel keeps one 16-bit count per id for the wedges in
    both graphs and lists the wedges in one graph only (through a changed
    pair) for their cross terms; a pivot with more of those than its list
    holds (112 entries for 200 vertices) takes them by walking its wedges
    again.  A dense 200-vertex graph with a batch changing half its edges
    sends every pivot to that kernel, most of them past the list."""
    n = 200
    keys = gen.er_graph(n, 4000, 43)
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    ins, dels = gen.random_batch(n, keys, 1000, 1000, 44)
    r = oracle.fdgc_step(rp, col, ins, dels, F0)
    with open_graph(gcb, n, rp, col) as g:
        g.set_tuning(**TUNINGS["c4_all_cluster"])
        assert g.count_static() == F0
        assert g.count_batch(ins, dels) == r["F"]
        assert g.counts() == F0
        assert g.apply(ins, dels) == r["F"]
        assert mod64(g.stats()["Ca"]) == mod64(r["Ca"])
        assert mod64(g.stats()["Cb"]) == mod64(r["Cb"])


def test_autotune_keeps_counts(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    ins, dels = gen.random_batch(n, keys, 500, 500, 32)
    r = oracle.fdgc_step(rp, col, ins, dels, F0)
    with open_graph(gcb, n, rp, col) as g:
        best, ms = g.autotune(reps=1)
        assert ms > 0 and best == g.tuning()
        assert g.count_static() == F0
        assert g.apply(ins, dels) == r["F"]


def _two_big_hubs():
    """Two hubs sharing 66,000 neighbours (degrees above 2^16, so one pair
    has 66,000 common neighbours) over a sparse background: the 4-cycle
    counters must switch to 32-bit halves."""
    n = 70000
    keys = set(int(k) for k in gen.er_graph(n, 40000, 41))
    for h in (0, 1):
        for v in range(2, 66002):
            keys.add((h << 32) | v)
    return n, np.array(sorted(keys), dtype=np.uint64)


def test_cluster_counters_switch_from_16_to_32_bits(gcb):
    """A hub one neighbour short of 2^16: the cluster kernel counts in the
    16-bit layout (a batch leaves one-graph wedges in its lists), then a
    batch lifts the hub past 2^16 and the same counter regions serve as
    32/32-bit counters; every count equals the oracle."""
    n = 70000
    keys = set(int(k) for k in gen.er_graph(n, 40000, 47) if (int(k) >> 32) > 1)
    for v in range(2, 65537):
        keys.add(v)  # (0, v)
    for v in range(2, 20002):
        keys.add((1 << 32) | v)
    keys = np.array(sorted(keys), dtype=np.uint64)
    rp, col = gen.csr_from_keys(n, keys)
    assert int(np.diff(rp).max()) == 65535
    og = oracle.OracleGraph(rp, col)
    rng = np.random.default_rng(48)
    with open_graph(gcb, n, rp, col) as g:
        g.set_tuning(**TUNINGS["c4_all_cluster"])
        assert g.counts() == og.F
        dels = np.array([(1, int(v)) for v in rng.choice(np.arange(2, 20002), 300, replace=False)], np.int32)
        ins = np.array([(int(a), int(b)) for a, b in rng.integers(2, n, size=(300, 2)) if a != b], np.int32)
        assert g.apply(ins, dels) == og.apply(ins, dels)["F"]
        ins2 = np.array([(0, 65537), (0, 65538), (0, 65539), (1, 65540)], np.int32)
        none = np.zeros((0, 2), np.int32)
        assert g.apply(ins2, none) == og.apply(ins2, none)["F"]
        assert g.count_static() == og.F


@pytest.mark.parametrize("opts", [dict(), dict(chunk_threshold=1)], ids=["cluster", "chunked"])
def test_hubs_beyond_16_bit_counts(gcb, opts):
    n, keys = _two_big_hubs()
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    ins, dels = gen.random_batch(n, keys, 300, 300, 42)
    r = oracle.fdgc_step(rp, col, ins, dels, F0)
    with open_graph(gcb, n, rp, col, **opts) as g:
        assert g.counts() == F0
        assert g.apply(ins, dels) == r["F"]
        assert mod64(g.stats()["sums_a"]) == mod64(r["sums_a"])


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_static_workload_graphs(gcb, name):
    n, keys = gen.workload_graph(name)
    rp, col = gen.csr_from_keys(n, keys)
    with open(os.path.join(GOLDEN_DIR, "workloads.json")) as f:
        gold = json.load(f)
    expect = gold["c1"]["static"] if name == "c1" else gold["c2"][0]["static"]
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts() == expect
        assert g.count_static() == expect


def test_empty_and_tiny_graphs(gcb):
    for n in (0, 1, 2, 3):
        rp = np.zeros(n + 1, np.int32)
        with open_graph(gcb, n, rp, np.zeros(0, np.int32)) as g:
            assert g.counts() == [0] * 6
    rp, col = csr_from_edges(3, [(0, 1), (1, 2)])
    with open_graph(gcb, 3, rp, col) as g:
        assert g.counts() == [0] * 6
        assert g.apply([(0, 2)], []) == [0] * 6


def test_malformed_csr_is_rejected(gcb):
    rp = np.array([0, 1, 1], np.int32)          # 0 -> 1 without 1 -> 0
    with pytest.raises(gcb.GCError) as ei:
        gcb.Graph(2, rp, np.array([1], np.int32))
    assert ei.value.code == gcb.GC_EINVAL
    rp = np.array([0, 2, 3], np.int32)          # repeated entry
    with pytest.raises(gcb.GCError):
        gcb.Graph(2, rp, np.array([1, 1, 0], np.int32))
    rp = np.array([0, 1, 2], np.int32)          # self-loop
    with pytest.raises(gcb.GCError):
        gcb.Graph(2, rp, np.array([0, 1], np.int32))


# ----------------------------------------------------------------- dynamic --

def check_step(g, r, stats):
    assert mod64(g.counts()) == mod64(r["F"])
    assert stats["Ca"] == r["Ca"] and stats["Cb"] == r["Cb"]
    assert stats["sums_a"] == r["sums_a"] and stats["sums_b"] == r["sums_b"]
    assert stats["region_vertices"] == r["region_vertices"]
    assert stats["edges_a"] == r["edges_a"] and stats["edges_b"] == r["edges_b"]
    assert stats["n_ins"] == r["n_ins"] and stats["n_del"] == r["n_del"]


def test_batch_workload_c1(gcb):
    """ER n=2,000 m=20,000: one batch of 200 deletions + 200 insertions."""
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.random_batch(n, keys, 200, 200, 1, ins_weighting="uniform")
    r = oracle.fdgc_step(rp, col, ins, dels, oracle.static_counts(rp, col), 3, "literal")
    with open(os.path.join(GOLDEN_DIR, "workloads.json")) as f:
        gold = json.load(f)["c1"]
    with open_graph(gcb, n, rp, col) as g:
        out = g.apply(ins, dels)
        st = g.stats()
        assert out == gold["after"] == r["F"]
        check_step(g, r, st)
        assert same_graph(g, r["row_ptr"], r["col"])
        assert g.count_static() == r["F"]


@pytest.mark.parametrize("ins_frac", [0.5, 1.0], ids=["fdgc", "igc"])
def test_stream_workload_c2(gcb, ins_frac):
    """Chung-Lu n=7,000 m=100,000: sequential batches of 1,000 and 10,000
    (50/50, or insert-only IGC), every step against the oracle."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts() == og.F
        for ins, dels in gen.batch_stream(n, keys, [1000, 10000, 1000, 10000], ins_frac, 2):
            r = og.apply(ins, dels)
            out = g.apply(ins, dels)
            assert out == r["F"]
            check_step(g, r, g.stats())
        assert same_graph(g, og.row_ptr, og.col)


def _dirty_batch(rng, n, edges, k_ins, k_del):
    es = list(edges)
    ins = [tuple(int(x) for x in rng.choice(n, 2, replace=False)) for _ in range(k_ins)]
    dels = [es[i] for i in rng.choice(len(es), min(k_del, len(es)), replace=False)] if es else []
    dels += [tuple(int(x) for x in rng.choice(n, 2, replace=False)) for _ in range(k_del // 3)]
    if ins and rng.random() < 0.5:
        dels.append(ins[0][::-1])
    if dels and rng.random() < 0.5:
        ins.append(dels[0])
    if ins:
        ins.append(ins[-1][::-1])
    return np.array(ins, np.int32).reshape(-1, 2), np.array(dels, np.int32).reshape(-1, 2)


def test_dirty_batches_on_random_graphs(gcb):
    """Repeats, reversed pairs, cancellations and no-ops, on graphs whose
    region is a strict subset of V (region-induced degrees matter)."""
    rng = np.random.default_rng(202)
    for trial in range(40):
        n = int(rng.integers(8, 200))
        edges = random_graph(rng, n, float(rng.uniform(0.005, 0.2)))
        rp, col = csr_from_edges(n, edges)
        og = oracle.OracleGraph(rp, col, variant="literal")
        with open_graph(gcb, n, rp, col) as g:
            for step in range(3):
                cur = edges_from_csr(og.row_ptr, og.col)
                ins, dels = _dirty_batch(rng, n, cur, int(rng.integers(0, 12)), int(rng.integers(0, 12)))
                r = og.apply(ins, dels)
                g.apply(ins, dels)
                st = g.stats()
                check_step(g, r, st)
                assert st["cancelled"] == r["cancelled"]
                assert st["noop_ins"] + st["noop_del"] == r["noops"]
                assert st["repeats"] == r["repeats"]
            assert same_graph(g, og.row_ptr, og.col)


def test_invalid_batches_change_nothing(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    with open_graph(gcb, n, rp, col) as g:
        F0 = g.counts()
        for ins, dels in (([(3, 3)], []), ([], [(0, n)]), ([(-1, 2)], []), ([(0, 1), (5, 5)], [])):
            with pytest.raises(gcb.GCError) as ei:
                g.apply(ins, dels)
            assert ei.value.code == gcb.GC_EINVAL
            assert g.counts() == F0
        assert same_graph(g, rp, col)


def test_empty_batch_and_all_noop_batch(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    with open_graph(gcb, n, rp, col) as g:
        F0 = g.counts()
        assert g.apply([], []) == F0
        assert g.stats()["region_vertices"] == 0
        existing = edges_from_csr(rp, col)[:50]
        assert g.apply(existing, []) == F0
        st = g.stats()
        assert st["noop_ins"] == 50 and st["n_ins"] == 0
        assert g.apply(existing[:10], existing[:10]) == F0
        assert g.stats()["cancelled"] == 10
        assert same_graph(g, rp, col)


def test_radius_two_gives_same_counts(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [1000, 5000], 0.5, 12)
    with open_graph(gcb, n, rp, col, region_hops=3) as g3, open_graph(gcb, n, rp, col, region_hops=2) as g2:
        for ins, dels in batches:
            assert g3.apply(ins, dels) == g2.apply(ins, dels)


def test_inverse_batch_restores_counts_and_graph(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.random_batch(n, keys, 3000, 2000, 77)
    with open_graph(gcb, n, rp, col) as g:
        F0 = g.counts()
        g.apply(ins, dels)
        assert g.counts() != F0
        assert g.apply(dels, ins) == F0
        assert same_graph(g, rp, col)


def test_row_growth_forces_relocation_and_relayout(gcb):
    """Insert many edges at a few vertices so rows outgrow their slack and the
    pool; the result must still equal the oracle."""
    n = 3000
    keys = gen.er_graph(n, 6000, 3)
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    rng = np.random.default_rng(9)
    with open_graph(gcb, n, rp, col, slack=0.05) as g:
        relayouts = 0
        for step in range(4):
            hubs = rng.choice(n, 3, replace=False)
            cur = set(int(k) for k in gen.keys_from_csr(og.row_ptr, og.col))
            ins = []
            for h in hubs:
                for v in rng.choice(n, 900, replace=False):
                    if v != h and ((min(h, v) << 32) | max(h, v)) not in cur:
                        ins.append((int(h), int(v)))
            ins = np.array(ins, np.int32)
            r = og.apply(ins, np.zeros((0, 2), np.int32))
            assert g.apply(ins, []) == r["F"]
            relayouts += g.stats()["relayouts"]
        assert same_graph(g, og.row_ptr, og.col)
        assert relayouts >= 1


def test_independent_batches_equal_fresh_copies(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    sizes = [10, 300, 5000, 40, 2000]
    batches = gen.batch_stream(n, keys, sizes, 0.5, 44, sequential=False)
    F0 = oracle.static_counts(rp, col)
    with open_graph(gcb, n, rp, col) as g:
        outs = g.apply_many(batches, independent=True)
        assert g.counts() == F0 and same_graph(g, rp, col)
    for (ins, dels), out in zip(batches, outs):
        assert out == oracle.fdgc_step(rp, col, ins, dels, F0)["F"]


def test_count_batch_is_a_what_if_query(gcb):
    """gc_count_batch returns the counts of G (+) B and leaves the graph and
    the maintained counts untouched; its stats carry C_a and C_b."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    with open_graph(gcb, n, rp, col) as g:
        for seed, (ni, nd) in enumerate([(700, 300), (0, 900), (1200, 0), (1, 1)]):
            ins, dels = gen.random_batch(n, keys, ni, nd, 60 + seed)
            r = oracle.fdgc_step(rp, col, ins, dels, F0)
            assert g.count_batch(ins, dels) == r["F"]
            st = g.stats()
            assert mod64(st["Ca"]) == mod64(r["Ca"]) and mod64(st["Cb"]) == mod64(r["Cb"])
            assert g.counts() == F0 and same_graph(g, rp, col)


def test_three_vertex_counts_follow_every_batch(gcb):
    """The maintained [2-paths, triangles] equal the oracle's static 3-vertex
    counts of the graph after each batch, in the plain and batched forms and
    for what-if batches (which leave them unchanged)."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [1500, 40, 3000, 700], 0.5, 71)
    og = oracle.OracleGraph(rp, col)
    expect = []
    for ins, dels in batches:
        og.apply(ins, dels)
        expect.append(oracle.static_counts3(og.row_ptr, og.col))
    base3 = oracle.static_counts3(rp, col)
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts3() == base3
        g.count_static()
        assert mod64(g.stats()["C3a"]) == base3
        g.count_batch(*batches[0])
        assert g.counts3() == base3
        for (ins, dels), e3 in zip(batches, expect):
            g.apply(ins, dels)
            assert g.counts3() == e3
    with open_graph(gcb, n, rp, col) as g:
        g.apply_many(batches)
        assert g.counts3() == expect[-1]


def test_delete_vertices(gcb):
    """Deleting vertices deletes their edges in one batch (adjacent listed
    vertices, repeats and a hub included); the counts equal the oracle's on
    the graph without those edges, and a re-inserted edge counts again."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    deg = np.diff(rp)
    hub = int(np.argmax(deg))
    a = int(col[rp[hub]])  # a neighbour of the hub: an edge between two listed vertices
    ids = [hub, a, 17, 17, 4000]
    drop = set(ids)
    kept = [(u, v) for u, v in edges_from_csr(rp, col) if u not in drop and v not in drop]
    rp2, col2 = csr_from_edges(n, kept)
    with open_graph(gcb, n, rp, col) as g:
        out = g.delete_vertices(ids)
        assert out == oracle.static_counts(rp2, col2) == g.counts()
        assert same_graph(g, rp2, col2)
        assert g.counts3() == oracle.static_counts3(rp2, col2)
        assert g.delete_vertices([]) == out
        with pytest.raises(gcb.GCError):
            g.delete_vertices([n])
        assert g.counts() == out
        back = [(hub, a)]
        rp3, col3 = csr_from_edges(n, kept + back)
        assert g.apply(np.array(back, np.int32), None) == oracle.static_counts(rp3, col3)


def test_add_vertices_then_connect_them(gcb):
    """New vertices start isolated (counts unchanged) and then take part in
    batches like any other: edges among themselves, to old vertices and to
    the hub; plain and batched forms, against the oracle on the grown graph."""
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    rng = np.random.default_rng(81)
    with open_graph(gcb, n, rp, col) as g:
        first = g.add_vertices(300)
        assert first == n and g.n == n + 300
        assert g.counts() == F0
        n2 = n + 300
        new = np.arange(n, n2)
        ins = [(int(a), int(b)) for a, b in zip(new[:-1], new[1:])]                 # a path of new vertices
        ins += [(int(v), int(rng.integers(0, n))) for v in new]                     # each to an old vertex
        ins += [(int(v), 0) for v in new[:50]]                                      # many to one old vertex
        ins = np.array(sorted({(min(a, b), max(a, b)) for a, b in ins if a != b}), np.int32)
        none = np.zeros((0, 2), np.int32)
        og = oracle.OracleGraph(*csr_from_edges(n2, edges_from_csr(rp, col)))
        r1 = og.apply(ins[:400], none)
        assert g.apply(ins[:400], none) == r1["F"]
        dels = np.array(edges_from_csr(og.row_ptr, og.col)[:30], np.int32)
        r2 = og.apply(ins[400:], dels)
        last = np.array([(int(new[0]), int(new[1]))], np.int32)
        r3 = og.apply(none, last)
        assert g.apply_many([(ins[400:], dels), (none, last)]) == [r2["F"], r3["F"]]
        assert same_graph(g, og.row_ptr, og.col)
        assert g.counts3() == oracle.static_counts3(og.row_ptr, og.col)
        with pytest.raises(gcb.GCError):
            g.apply(np.array([[0, n2]], np.int32), none)


def test_sequential_batches_call_equals_single_calls(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [700, 50, 4000], 0.5, 45)
    with open_graph(gcb, n, rp, col) as g1, open_graph(gcb, n, rp, col) as g2:
        outs = g1.apply_many(batches)
        for (ins, dels), out in zip(batches, outs):
            assert g2.apply(ins, dels) == out


def test_device_resident_batch(gcb):
    torch = pytest.importorskip("torch")
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.random_batch(n, keys, 800, 600, 5)
    r = oracle.fdgc_step(rp, col, ins, dels, oracle.static_counts(rp, col))
    ti = torch.from_numpy(ins).cuda()
    td = torch.from_numpy(dels).cuda()
    torch.cuda.synchronize()
    with open_graph(gcb, n, rp, col) as g:
        out = gcb.gc_apply_batch_device(g.h, ti.data_ptr(), ins.shape[0], td.data_ptr(), dels.shape[0])
        assert out == r["F"]


# -------------------------------------------------------------- full size --

def _large_gold():
    p = os.path.join(GOLDEN_DIR, "workloads_large.json")
    if not os.path.exists(p):
        pytest.skip("workloads_large.json not generated")
    with open(p) as f:
        return json.load(f)


@pytest.mark.slow
def test_fullsize_c3_static_and_first_batch(gcb):
    """Chung-Lu n=1.6M m=30M: static count and one 100,000-update batch
    against stored oracle results, plus Lemma 2 on the device."""
    gold = _large_gold()["c3"]
    n, keys = gen.workload_graph("c3")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.batch_stream(n, keys, [100000], 0.6, 3)[0]
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts() == gold["static"]
        out = g.apply(ins, dels)
        st = g.stats()
        assert out == gold["after"]
        assert st["Ca"] == gold["Ca"] and st["Cb"] == gold["Cb"]
        assert st["region_vertices"] == gold["region_vertices"]
        assert g.count_static() == out


@pytest.mark.slow
@pytest.mark.parametrize("local", [0, 512], ids=["region", "local_up_to_512"])
def test_fullsize_c4_independent_batches(gcb, local):
    """Chung-Lu n=2.4M m=5M with 40k-degree hubs: independent batches on one
    snapshot against stored oracle results (with the small ones also through
    the edge-local delta)."""
    gold = _large_gold()["c4"]
    n, keys = gen.workload_graph("c4")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, gold["sizes"], 0.5, 4, sequential=False)
    with open_graph(gcb, n, rp, col, local_max_pairs=local) as g:
        assert g.counts() == gold["static"]
        outs = g.apply_many(batches, independent=True)
        for out, b in zip(outs, gold["batches"]):
            assert out == b["after"]


@pytest.mark.slow
def test_fullsize_c3_local_batches_keep_counts_of_the_graph(gcb):
    """Chung-Lu n=1.6M m=30M: sequential batches of the paper's sizes through
    the edge-local delta; the maintained counts equal a recount of the
    updated graph, and a twin handle on the region form agrees batch by
    batch."""
    n, keys = gen.workload_graph("c3")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [10, 100, 1000, 10, 100], 0.7, 77)
    with open_graph(gcb, n, rp, col, local_max_pairs=1 << 30) as gl, open_graph(gcb, n, rp, col) as gr:
        for ins, dels in batches:
            out = gl.apply(ins, dels)
            assert gl.stats()["path"] == 1
            assert out == gr.apply(ins, dels)
        assert gl.count_static() == gl.counts()
        # the oracle's count of the final edge set (Lemma 2: the maintained
        # counts are those of the updated graph)
        gold = _large_gold().get("c3_local_stream")
        if gold is not None:
            assert gold["sizes"] == [10, 100, 1000, 10, 100] and gold["seed"] == 77
            assert gl.counts() == gold["final"]
            assert gl.num_edges() == gold["edges"]


@pytest.mark.slow
def test_fullsize_c3_ten_thousand_pairs_through_the_edge_local_delta(gcb):
    """One 10,000-update batch on the 1.6M-vertex graph through the edge-local
    delta (the autotuner keeps batches up to 16,384 pairs on it there): the
    counts equal the oracle's count of the updated graph, and the region
    form on a twin handle agrees."""
    gold = _large_gold().get("c3_local_10k")
    if gold is None:
        pytest.skip("c3_local_10k not in workloads_large.json")
    n, keys = gen.workload_graph("c3")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.batch_stream(n, keys, [gold["size"]], 0.7, gold["seed"])[0]
    with open_graph(gcb, n, rp, col, local_max_pairs=1 << 30) as gl, open_graph(gcb, n, rp, col) as gr:
        out = gl.apply(ins, dels)
        assert gl.stats()["path"] == 1
        assert out == gold["final"]
        assert gr.apply(ins, dels) == out
        assert gl.num_edges() == gold["edges"]


def _c5_gold():
    p = os.path.join(GOLDEN_DIR, "workloads_c5.json")
    if not os.path.exists(p):
        pytest.skip("workloads_c5.json not generated")
    with open(p) as f:
        return json.load(f)


@pytest.mark.slow
@pytest.mark.parametrize("gi", [0, 7], ids=["n100k_m1M", "n4.8M_m69M"])
def test_fullsize_c5_graph_static_and_batch(gcb, gi):
    """The smallest and the largest graph of the serving workload (Chung-Lu,
    1M and 69M edges): static count and one 100,000-update batch (70%
    insertions) against stored oracle results, with the counts of G_a and G_b
    and the region size."""
    gold = _c5_gold().get(f"g{gi}")
    if gold is None:
        pytest.skip(f"graph {gi} of the serving workload not in workloads_c5.json")
    p = gen.c5_graph_params()[gi]
    assert gold["params"] == p
    n, keys = gen.workload_graph(p)
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.batch_stream(n, keys, [100000], 0.7, 500 + gi)[0]
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts() == gold["static"]
        out = g.apply(ins, dels)
        st = g.stats()
        assert out == gold["after"]
        assert st["Ca"] == gold["Ca"] and st["Cb"] == gold["Cb"]
        assert st["region_vertices"] == gold["region_vertices"]
        assert (st["n_ins"], st["n_del"]) == (gold["n_ins"], gold["n_del"])
        assert g.count_static() == out


@pytest.mark.slow
def test_fullsize_c5_stream_plain_and_served(gcb):
    """A sequential stream of 5 batches (100..100,000 updates, log-uniform)
    on the 1M-edge serving graph: the counts after every batch equal the
    oracle's, through gc_apply_batch and through the request server."""
    gold = _c5_gold().get("g0_stream")
    if gold is None:
        pytest.skip("stream of the serving workload not in workloads_c5.json")
    n, keys = gen.workload_graph(gen.c5_graph_params()[0])
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, gold["sizes"], 0.7, gold["seed"])
    expect = [s["after"] for s in gold["steps"][1:]]
    with open_graph(gcb, n, rp, col) as g:
        assert g.counts() == gold["steps"][0]["static"]
        assert [g.apply(i, d) for i, d in batches] == expect
    with open_graph(gcb, n, rp, col) as g:
        with gcb.Server([g], slots=2) as srv:
            tickets = [srv.submit(0, i, d) for i, d in batches]
            res = [srv.wait(t) for t in tickets]
        assert all(r["status"] == 0 for r in res)
        assert [r["counts"] for r in res] == expect
        assert g.counts() == expect[-1]


# ----------------------------------------------------------- batched form --

def test_batched_run_that_outgrows_the_pool(gcb):
    """A captured multi-batch run whose commits outgrow the adjacency pool
    mid-run (the run pauses, the pool grows, the run resumes) still matches
    the oracle batch by batch."""
    n = 3000
    keys = gen.er_graph(n, 6000, 3)
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    rng = np.random.default_rng(19)
    batches, expect = [], []
    for step in range(5):
        hubs = rng.choice(n, 3, replace=False)
        cur = set(int(k) for k in gen.keys_from_csr(og.row_ptr, og.col))
        ins = []
        for h in hubs:
            for v in rng.choice(n, 900, replace=False):
                kk = (min(h, v) << 32) | max(h, v)
                if v != h and kk not in cur:
                    cur.add(kk)
                    ins.append((int(h), int(v)))
        edges = edges_from_csr(og.row_ptr, og.col)
        dels = np.array([edges[i] for i in rng.choice(len(edges), 50, replace=False)], np.int32)
        ins = np.array(ins, np.int32)
        batches.append((ins, dels))
        expect.append(og.apply(ins, dels)["F"])
    with open_graph(gcb, n, rp, col, slack=0.05) as g:
        outs = g.apply_many(batches)
        assert outs == expect
        assert g.stats()["relayouts"] >= 1
        assert same_graph(g, og.row_ptr, og.col)
        assert g.count_static() == expect[-1]


def test_batched_run_that_relocates_hub_rows_repeatedly(gcb):
    """Few insertions into many nearly full hub rows: every batch relocates
    whole rows, more than the pool grown ahead of the run can take, so the
    run halts and resumes mid-way; results still match the oracle."""
    n = 3000
    rng = np.random.default_rng(29)
    keys = set(int(k) for k in gen.er_graph(n, 3000, 28))
    hubs = list(range(20))
    for h in hubs:
        for v in rng.choice(np.arange(20, n), 500, replace=False):
            keys.add((h << 32) | int(v))
    keys = np.array(sorted(keys), dtype=np.uint64)
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    batches, expect = [], []
    for step in range(6):
        cur = set(int(k) for k in gen.keys_from_csr(og.row_ptr, og.col))
        ins = []
        for h in hubs:
            added = 0
            for v in rng.permutation(np.arange(20, n)):
                kk = (h << 32) | int(v)
                if kk not in cur:
                    cur.add(kk)
                    ins.append((h, int(v)))
                    added += 1
                    if added == 30:
                        break
        edges = edges_from_csr(og.row_ptr, og.col)
        dels = np.array([edges[i] for i in rng.choice(len(edges), 20, replace=False)], np.int32)
        ins = np.array(ins, np.int32)
        batches.append((ins, dels))
        expect.append(og.apply(ins, dels)["F"])
    with open_graph(gcb, n, rp, col, slack=0.05) as g:
        outs = g.apply_many(batches)
        assert outs == expect
        assert g.stats()["relayouts"] >= 2
        assert same_graph(g, og.row_ptr, og.col)


def test_device_batched_api_equals_plain(gcb):
    torch = pytest.importorskip("torch")
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [1000, 10, 5000, 300], 0.5, 71)
    pairs, desc, off = [], [], 0
    for ins, dels in batches:
        desc.append((off, len(ins), off + len(ins), len(dels)))
        pairs += [ins, dels]
        off += len(ins) + len(dels)
    d_pairs = torch.from_numpy(np.ascontiguousarray(np.concatenate(pairs).astype(np.int32))).cuda()
    torch.cuda.synchronize()
    with open_graph(gcb, n, rp, col) as g1, open_graph(gcb, n, rp, col) as g2:
        plain = [g1.apply(i, d) for i, d in batches]
        got = gcb.gc_apply_batches_device(g2.h, d_pairs.data_ptr(), desc)
        assert got == plain
        assert g2.counts() == g1.counts() and g2.num_edges() == g1.num_edges()
    with open_graph(gcb, n, rp, col) as g3:
        ind = gcb.gc_apply_batches_device(g3.h, d_pairs.data_ptr(), desc, independent=True)
        F0 = g3.counts()
    for (ins, dels), out in zip(batches, ind):
        assert out == oracle.fdgc_step(rp, col, ins, dels, F0)["F"]


def test_batched_runs_reuse_and_recapture(gcb):
    """Runs of different shapes on one handle (the captured graph is reused or
    captured again) agree with the plain form."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    runs = [gen.batch_stream(n, keys, sizes, 0.5, 80 + i)
            for i, sizes in enumerate([[200, 200], [150, 180], [20000], [5, 6, 7]])]
    with open_graph(gcb, n, rp, col) as gb, open_graph(gcb, n, rp, col) as gp:
        for run in runs:
            assert gb.apply_many(run) == [gp.apply(i, d) for i, d in run]
            assert gb.counts() == gp.counts()


def test_batched_invalid_pair_changes_nothing(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    with open_graph(gcb, n, rp, col) as g:
        F0 = g.counts()
        ok = gen.random_batch(n, keys, 10, 10, 3)
        with pytest.raises(gcb.GCError):
            g.apply_many([ok, ([(1, 1)], [])])
        assert g.counts() == F0 and same_graph(g, rp, col)
