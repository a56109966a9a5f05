"""Per-vertex graphlet counts (gc_vertex_counts) against the oracle, bit-exact,
on random, planted and workload graphs and after batches; at larger sizes
the sum over vertices must be four times the global counts."""
import numpy as np
import pytest

import oracle
from synth import gen
from gc_testutil import csr_from_edges, random_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gcb():
    from paper_2308_14493_gb300 import gc as binding

    binding.load()
    return binding


def _check(g, rp, col):
    got = g.vertex_counts().astype(np.int64).tolist()
    assert got == oracle.vertex_counts(rp, col)


def test_vertex_counts_random_graphs(gcb):
    rng = np.random.default_rng(31)
    for trial in range(25):
        n = int(rng.integers(4, 90))
        edges = random_graph(rng, n, float(rng.uniform(0.03, 0.8)))
        rp, col = csr_from_edges(n, edges)
        with gcb.Graph(n, rp, col) as g:
            _check(g, rp, col)


def test_vertex_counts_hubs_and_cliques(gcb):
    n = 300
    edges = {(0, v) for v in range(1, n)}                       # a hub
    edges |= {(a, b) for a in range(1, 15) for b in range(a + 1, 15)}  # a clique at the hub
    edges |= {(v, v + 1) for v in range(20, n - 1)}             # a path through its leaves
    edges |= {(a, b) for a in range(100, 110) for b in range(200, 210)}  # K_{10,10}: many 4-cycles
    rp, col = csr_from_edges(n, sorted(edges))
    with gcb.Graph(n, rp, col) as g:
        _check(g, rp, col)


def test_vertex_counts_workload_and_after_batches(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=50) as g:
        _check(g, rp, col)
        for i, size in enumerate([20, 400]):
            ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), size // 2, size - size // 2, 40 + i)
            og.apply(ins, dels)
            g.apply(ins, dels)
            _check(g, og.row_ptr, og.col)
        assert g.counts() == og.F   # the maintained counts are untouched


@pytest.mark.parametrize("name", ["c2", "hub"])
def test_vertex_counts_sum_to_four_times_the_counts(gcb, name):
    if name == "c2":
        n, keys = gen.workload_graph("c2")
    else:
        n, keys = 200_000, gen.chung_lu_graph(200_000, 2_000_000, 1.9, 30_000.0, 3)
    rp, col = gen.csr_from_keys(n, keys)
    with gcb.Graph(n, rp, col) as g:
        v = g.vertex_counts()
        tot = [int(x) for x in v.astype(object).sum(axis=0)]
        assert tot == [4 * x for x in g.counts()]
        deg = np.diff(rp)
        assert np.all(v[deg == 0] == 0)


def test_vertex_orbits_random_and_planted(gcb):
    rng = np.random.default_rng(77)
    cases = []
    for trial in range(15):
        n = int(rng.integers(4, 80))
        cases.append((n, random_graph(rng, n, float(rng.uniform(0.03, 0.8)))))
    n = 200
    edges = {(0, v) for v in range(1, n)} | {(a, b) for a in range(1, 12) for b in range(a + 1, 12)}
    edges |= {(v, v + 1) for v in range(20, n - 1)} | {(a, b) for a in range(100, 108) for b in range(150, 158)}
    cases.append((n, sorted(edges)))
    for n, edges in cases:
        rp, col = csr_from_edges(n, edges)
        with gcb.Graph(n, rp, col) as g:
            orb = g.vertex_orbits().astype(np.int64)
            assert orb.tolist() == oracle.vertex_orbits(rp, col)
            per = g.vertex_counts().astype(np.int64)
            sums = np.stack([orb[:, 0] + orb[:, 1], orb[:, 2] + orb[:, 3], orb[:, 4],
                             orb[:, 5] + orb[:, 6] + orb[:, 7], orb[:, 8] + orb[:, 9], orb[:, 10]], axis=1)
            assert np.array_equal(per, sums)


@pytest.mark.parametrize("heavy_min", [0, 1, 40])
def test_vertex_orbits_every_4cycle_walk(gcb, heavy_min):
    """The 4-cycle walk of the local counts: every pivot on the per-CTA
    arrays (0), every pivot with lower neighbours in the grouped L2 walk
    (1), and a split between the two (40)."""
    rng = np.random.default_rng(90 + heavy_min)
    cases = [(n, random_graph(rng, n, float(rng.uniform(0.05, 0.7)))) for n in (12, 40, 150)]
    n = 300
    edges = {(0, v) for v in range(1, n)} | {(a, b) for a in range(1, 15) for b in range(a + 1, 15)}
    edges |= {(a, b) for a in range(100, 110) for b in range(200, 210)}
    cases.append((n, sorted(edges)))
    for n, edges in cases:
        rp, col = csr_from_edges(n, edges)
        with gcb.Graph(n, rp, col) as g:
            g.set_tuning(local_c4_heavy_min=heavy_min)
            assert g.tuning()["local_c4_heavy_min"] == heavy_min
            assert g.vertex_orbits().astype(np.int64).tolist() == oracle.vertex_orbits(rp, col)
