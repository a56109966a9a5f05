"""Per-edge graphlet and orbit counts (gc_edge_counts, gc_edge_orbits)
against the oracle, bit-exact, on random, planted and workload graphs and
after batches; at full workload sizes on a sample of edges the oracle
counts one by one, and through the sums over edges, which give the global
counts times the edges of each graphlet in each orbit."""
import numpy as np
import pytest

import oracle
from synth import gen
from gc_testutil import csr_from_edges, random_graph

pytestmark = pytest.mark.gpu

# edges of each graphlet in each edge orbit: 3-path 2 ends + 1 middle,
# 3-star 3, 4-cycle 4, tailed triangle 1 + 1 + 2, diamond 4 outer + 1 chord, 4-clique 6
PER_ORBIT = [(0, 2), (0, 1), (1, 3), (2, 4), (3, 1), (3, 1), (3, 2), (4, 4), (4, 1), (5, 6)]


@pytest.fixture(scope="module")
def gcb():
    from paper_2308_14493_gb300 import gc as binding

    binding.load()
    return binding


def _sorted_edges(rp, col):
    src = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    keep = src < col
    return np.stack([src[keep], np.asarray(col)[keep]], axis=1).astype(np.int32)


def _check(g, rp, col):
    edges, orb = g.edge_orbits()
    keys, rows = oracle.edge_orbits(rp, col)
    assert edges.tolist() == [list(k) for k in keys]
    assert orb.astype(np.int64).tolist() == rows
    e6, per = g.edge_counts()
    assert np.array_equal(e6, edges)
    o = orb.astype(np.int64)
    sums = np.stack([o[:, 0] + o[:, 1], o[:, 2], o[:, 3], o[:, 4] + o[:, 5] + o[:, 6], o[:, 7] + o[:, 8], o[:, 9]],
                    axis=1)
    assert np.array_equal(per.astype(np.int64), sums)


def test_edge_orbits_random_graphs(gcb):
    rng = np.random.default_rng(52)
    for trial in range(25):
        n = int(rng.integers(4, 90))
        edges = random_graph(rng, n, float(rng.uniform(0.03, 0.8)))
        rp, col = csr_from_edges(n, edges)
        with gcb.Graph(n, rp, col) as g:
            _check(g, rp, col)


def test_edge_orbits_hubs_cliques_and_bicliques(gcb):
    n = 300
    edges = {(0, v) for v in range(1, n)}                                  # a hub
    edges |= {(a, b) for a in range(1, 15) for b in range(a + 1, 15)}      # a clique at the hub
    edges |= {(v, v + 1) for v in range(20, n - 1)}                        # a path through its leaves
    edges |= {(a, b) for a in range(100, 110) for b in range(200, 210)}    # K_{10,10}: many 4-cycles
    rp, col = csr_from_edges(n, sorted(edges))
    with gcb.Graph(n, rp, col) as g:
        _check(g, rp, col)


def test_edge_orbits_empty_and_tiny_graphs(gcb):
    for n, edges in ((1, []), (5, []), (2, [(0, 1)]), (4, [(0, 1), (2, 3)]), (6, [(4, 5)])):
        rp, col = csr_from_edges(n, edges)
        with gcb.Graph(n, rp, col) as g:
            _check(g, rp, col)


def test_edge_orbits_workload_and_after_batches(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=50) as g:
        _check(g, rp, col)
        for i, size in enumerate([20, 400]):   # the edge-local form, then the region form
            ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), size // 2, size - size // 2,
                                         60 + i)
            og.apply(ins, dels)
            g.apply(ins, dels)
            _check(g, og.row_ptr, og.col)
        assert g.counts() == og.F   # the maintained counts are untouched


@pytest.mark.parametrize("name", ["c2", "hub"])
def test_edge_orbits_full_size_sample_and_sums(gcb, name):
    if name == "c2":
        n, keys = gen.workload_graph("c2")
    else:
        n, keys = 200_000, gen.chung_lu_graph(200_000, 2_000_000, 1.9, 30_000.0, 3)
    rp, col = gen.csr_from_keys(n, keys)
    with gcb.Graph(n, rp, col) as g:
        edges, orb = g.edge_orbits()
        assert np.array_equal(edges, _sorted_edges(rp, col))
        tot = [int(x) for x in orb.astype(object).sum(axis=0)]
        F = g.counts()
        assert tot == [mult * F[k] for k, mult in PER_ORBIT]
        # a sample of rows, uniform plus the edges of the largest hub (the
        # oracle walks the hub's neighbourhood for each of those)
        rng = np.random.default_rng(9)
        n_uni, n_hub = (300, 20) if name == "c2" else (60, 8)
        pick = set(rng.choice(len(edges), size=n_uni, replace=False).tolist())
        hub = int(np.argmax(np.diff(rp)))
        at_hub = np.nonzero((edges[:, 0] == hub) | (edges[:, 1] == hub))[0]
        pick |= set(rng.choice(at_hub, size=min(n_hub, at_hub.size), replace=False).tolist())
        pick = sorted(pick)
        keys_s, rows = oracle.edge_orbits(rp, col, [tuple(edges[i]) for i in pick])
        assert [list(k) for k in keys_s] == edges[pick].tolist()
        assert orb[pick].astype(np.int64).tolist() == rows


@pytest.mark.parametrize("heavy_min", [0, 1, 40])
def test_edge_orbits_every_4cycle_walk(gcb, heavy_min):
    """Per-edge counts with every pivot on the per-CTA arrays (0), every
    pivot in the grouped L2 walk (1), and a split (40)."""
    rng = np.random.default_rng(70 + heavy_min)
    cases = [(n, random_graph(rng, n, float(rng.uniform(0.05, 0.7)))) for n in (12, 40, 150)]
    n = 300
    edges = {(0, v) for v in range(1, n)} | {(a, b) for a in range(1, 15) for b in range(a + 1, 15)}
    edges |= {(a, b) for a in range(100, 110) for b in range(200, 210)}
    cases.append((n, sorted(edges)))
    for n, edges in cases:
        rp, col = csr_from_edges(n, edges)
        with gcb.Graph(n, rp, col) as g:
            g.set_tuning(local_c4_heavy_min=heavy_min)
            _check(g, rp, col)
