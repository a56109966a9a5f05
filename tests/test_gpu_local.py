"""Parity of the edge-local delta (gc_options.local_max_pairs) with the oracle.

Small batches on graphs with hubs, cliques and dense cores, dirty batches
(repeats, cancellations, no-ops), what-if batches, and a batch whose rows
outgrow the first local scratch.  Every result must equal the oracle's
Algorithm 2 step bit-exactly; the path actually taken is read back from the
batch record (stats['path'] == 1).
"""
import numpy as np
import pytest

import oracle
from synth import gen
from gc_testutil import csr_from_edges, edges_from_csr, random_graph

pytestmark = pytest.mark.gpu

ALWAYS = 1 << 30  # local_max_pairs: every batch takes the edge-local path
NONE = np.zeros((0, 2), np.int32)


@pytest.fixture(scope="module")
def gcb():
    from paper_2308_14493_gb300 import gc as binding

    binding.load()
    return binding


def mod64(xs):
    return [int(x) & 0xFFFFFFFFFFFFFFFF for x in xs]


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


def _step(g, og, ins, dels):
    r = og.apply(ins, dels)
    out = g.apply(ins, dels)
    st = g.stats()
    assert st["path"] == 1
    assert out == mod64(r["F"])
    # the local record holds the deltas: C_a - C_b of the region recount
    assert st["Ca"] == [a - b for a, b in zip(r["Ca"], r["Cb"])]
    assert st["Cb"] == [0] * 6
    assert st["n_ins"] == r["n_ins"] and st["n_del"] == r["n_del"]
    return r


def test_local_dirty_batches_on_random_graphs(gcb):
    rng = np.random.default_rng(404)
    for trial in range(30):
        n = int(rng.integers(6, 120))
        edges = random_graph(rng, n, float(rng.uniform(0.02, 0.6)))
        rp, col = csr_from_edges(n, edges)
        og = oracle.OracleGraph(rp, col, variant="literal")
        with gcb.Graph(n, rp, col, local_max_pairs=ALWAYS) as g:
            for step in range(4):
                cur = edges_from_csr(og.row_ptr, og.col)
                ins, dels = _dirty_batch(rng, n, cur, int(rng.integers(0, 15)), int(rng.integers(0, 15)))
                _step(g, og, ins, dels)
                assert g.counts3() == oracle.static_counts3(og.row_ptr, og.col)
            grp, gcol = g.export_csr()
            assert np.array_equal(grp.astype(np.int64), og.row_ptr) and np.array_equal(gcol, og.col)


def test_local_batches_inside_cliques(gcb):
    """Many pairs of one batch inside the same 4-cliques and 4-cycles: each
    such subgraph must be counted once (at its smallest changed pair)."""
    rng = np.random.default_rng(7)
    n = 40
    full = [(a, b) for a in range(14) for b in range(a + 1, 14)]           # K_14 core
    ring = [(i, i + 1) for i in range(14, n - 1)] + [(13, 14), (0, n - 1)]  # and a path around it
    for trial in range(6):
        drop = [full[i] for i in rng.choice(len(full), size=25, replace=False)]
        base = sorted(set(full + ring) - set(drop))
        rp, col = csr_from_edges(n, base)
        og = oracle.OracleGraph(rp, col, variant="literal")
        with gcb.Graph(n, rp, col, local_max_pairs=ALWAYS) as g:
            _step(g, og, np.array(drop, np.int32), NONE)                     # insert them all back
            dels = [full[i] for i in rng.choice(len(full), size=30, replace=False)]
            _step(g, og, NONE, np.array(dels, np.int32))                     # delete 30 clique edges
            mix_i = [e for e in drop[:10]]
            mix_d = [e for e in full if e not in dels][:10]
            _step(g, og, np.array(mix_i, np.int32), np.array(mix_d, np.int32))


def test_local_and_region_paths_agree_on_c2(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    sizes = [1, 2, 5, 10, 30, 100, 300, 1000]
    batches = gen.batch_stream(n, keys, sizes, 0.5, 31)
    with gcb.Graph(n, rp, col, local_max_pairs=ALWAYS) as gl, gcb.Graph(n, rp, col) as gr:
        for ins, dels in batches:
            r = _step(gl, og, ins, dels)
            assert gr.apply(ins, dels) == mod64(r["F"])
            assert gr.stats()["path"] == 0
        assert gl.counts3() == gr.counts3() == oracle.static_counts3(og.row_ptr, og.col)


def test_local_threshold_picks_the_path(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=64) as g:
        for size, path in ((64, 1), (65, 0), (3, 1)):
            ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), size - size // 2, size // 2, size)
            r = og.apply(ins, dels)
            assert g.apply(ins, dels) == mod64(r["F"])
            assert g.stats()["path"] == path


def test_local_what_if_batches_leave_the_graph(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=ALWAYS) as g:
        for seed in range(5):
            ins, dels = gen.random_batch(n, keys, 20, 20, 100 + seed)
            r = oracle.fdgc_step(rp, col, ins, dels, F0, 3)
            assert g.count_batch(ins, dels) == mod64(r["F"])
            assert g.stats()["path"] == 1
            assert g.counts() == mod64(F0)
        assert g.count_static() == mod64(F0)


def test_local_empty_and_noop_batches(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    with gcb.Graph(n, rp, col, local_max_pairs=ALWAYS) as g:
        F0 = g.counts()
        assert g.apply([], []) == F0
        existing = edges_from_csr(rp, col)[:20]
        assert g.apply(existing, []) == F0
        assert g.apply(existing[:5], existing[:5]) == F0
        with pytest.raises(gcb.GCError):
            g.apply([(0, n)], [])
        assert g.counts() == F0


def test_local_scratch_grows_for_a_hub(gcb):
    """A hub of 1.3M neighbours: the union rows of a batch at the hub exceed
    the first local scratch (2^20 entries); the batch is re-run with larger
    scratch and still matches the oracle."""
    L = 1_300_000
    n = L + 1
    hub = L
    rng = np.random.default_rng(3)
    edges = [(i, hub) for i in range(L)] + [(i, i + 1) for i in range(0, L - 1, 2)]
    rp, col = csr_from_edges(n, edges)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=ALWAYS) as g:
        assert g.counts() == mod64(og.F)
        ins = [(int(a), int(b)) for a, b in rng.integers(0, L, size=(6, 2)) if a != b]
        dels = [(0, hub), (5, hub), (2, 3)]
        _step(g, og, np.array(ins, np.int32), np.array(dels, np.int32))
        assert g.stats()["region_entries"] > (1 << 20)


def test_local_batches_at_hubs_beyond_the_staged_hash(gcb):
    """Hubs of 30,000 and 20,000 neighbours, rows longer than the
    shared-memory hash of the local kernels (12,288 entries), so their
    lookups search the rows in global memory; batches concentrated at the
    hubs, with the pair of hubs inserted then deleted, match the oracle step
    by step."""
    n = 40000
    rng = np.random.default_rng(7)
    edges = set()
    for h, k in ((0, 30000), (1, 20000)):
        for v in rng.choice(np.arange(2, n), k, replace=False):
            edges.add((h, int(v)))
    for a, b in rng.integers(2, n, size=(60000, 2)):
        if a != b:
            edges.add((int(min(a, b)), int(max(a, b))))
    rp, col = csr_from_edges(n, edges)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=ALWAYS) as g:
        assert g.counts() == mod64(og.F)
        for step in range(2):
            cur = sorted(edges_from_csr(og.row_ptr, og.col))
            hub_edges = [e for e in cur if e[0] < 2 and e[1] >= 2]
            ins = [(int(h), int(v)) for h, v in zip(rng.integers(0, 2, 150), rng.integers(2, n, 150))]
            ins += [(int(a), int(b)) for a, b in rng.integers(2, n, size=(50, 2)) if a != b]
            dels = [hub_edges[i] for i in rng.choice(len(hub_edges), 100, replace=False)]
            dels += [cur[i] for i in rng.choice(len(cur), 50, replace=False)]
            # the pair of hubs: its 4-cycle probes look up the other hub's row
            (ins if step == 0 else dels).append((0, 1))
            _step(g, og, np.array(ins, np.int32), np.array(dels, np.int32))


def test_local_after_region_batches_and_recount(gcb):
    """The maintained triangle sums are valid after open and after a static
    recount, stale after a committed region batch (the local path then
    intersects every edge at the endpoints); every mix stays exact."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=100) as g:
        def step(size, path, seed):
            ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), size - size // 3, size // 3, seed)
            r = og.apply(ins, dels)
            assert g.apply(ins, dels) == mod64(r["F"])
            assert g.stats()["path"] == path
        for i, (size, path) in enumerate([(40, 1), (90, 1), (500, 0), (30, 1), (60, 1)]):
            step(size, path, 60 + i)
        assert g.count_static() == mod64(og.F)
        for i in range(4):
            step(20 + 20 * i, 1, 80 + i)
            # what-if batches leave the sums as they are
            ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), 7, 7, 90 + i)
            r = oracle.fdgc_step(og.row_ptr, og.col, ins, dels, og.F, 3)
            assert g.count_batch(ins, dels) == mod64(r["F"])
        assert g.counts3() == oracle.static_counts3(og.row_ptr, og.col)


def test_local_after_adding_vertices(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    with gcb.Graph(n, rp, col, local_max_pairs=1 << 30) as g:
        first = g.add_vertices(5)
        assert first == n
        rp2 = np.concatenate([rp, np.full(5, rp[-1], rp.dtype)])
        og = oracle.OracleGraph(rp2, col)
        ins = np.array([(n, 0), (n, 1), (n + 1, 0), (n + 1, n), (n + 2, 3), (0, 1)], np.int32)
        _step(g, og, ins, NONE)
        _step(g, og, np.array([(n + 3, n + 4), (n + 4, 0), (n + 3, 0)], np.int32), np.array([(n, 1)], np.int32))


@pytest.mark.parametrize("independent", [False, True], ids=["sequential", "independent"])
def test_batched_run_routes_small_batches_to_the_local_path(gcb, independent):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    sizes = [5, 2000, 40, 60, 3000, 1, 800, 10]
    batches = gen.batch_stream(n, keys, sizes, 0.5, 55, sequential=not independent)
    og = oracle.OracleGraph(rp, col)
    F0 = og.F
    expect = []
    for ins, dels in batches:
        if independent:
            expect.append(mod64(oracle.fdgc_step(rp, col, ins, dels, F0, 3)["F"]))
        else:
            expect.append(mod64(og.apply(ins, dels)["F"]))
    with gcb.Graph(n, rp, col, local_max_pairs=100) as g:
        got = g.apply_many(batches, independent=independent)
        assert [list(map(int, o)) for o in got] == expect
        if independent:
            assert g.counts() == mod64(F0)
        else:
            assert g.counts() == expect[-1]
            assert g.counts3() == oracle.static_counts3(og.row_ptr, og.col)


def test_autotune_sets_a_local_threshold_and_keeps_counts(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col) as g:
        tuning, _ = g.autotune(reps=1)
        thr = tuning["local_max_pairs"]
        assert thr >= 0 and g.tuning()["local_max_pairs"] == thr
        for i, size in enumerate([4, 30, 300, 3000]):
            ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), size // 2, size - size // 2, 500 + i)
            r = og.apply(ins, dels)
            assert g.apply(ins, dels) == mod64(r["F"])
            assert g.stats()["path"] == (1 if size <= thr else 0)
        g.set_tuning(local_max_pairs=0)
        ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), 2, 2, 600)
        r = og.apply(ins, dels)
        assert g.apply(ins, dels) == mod64(r["F"])
        assert g.stats()["path"] == 0


def test_triangle_sums_through_region_runs_and_toggles(gcb):
    """Region batches keep the sums while the local form is enabled (plain
    and batched runs); with it disabled they go stale, and a later local
    batch still counts right (it intersects every edge at its endpoints)."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=50) as g:
        def mk(size, seed):
            return gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), size - size // 2, size // 2, seed)

        def step(size, seed, path):
            ins, dels = mk(size, seed)
            r = og.apply(ins, dels)
            assert g.apply(ins, dels) == mod64(r["F"])
            assert g.stats()["path"] == path

        step(400, 1, 0)
        step(30, 2, 1)
        # a batched run: region sub-runs between local batches
        run = [mk(300, 3)]
        r1 = og.apply(*run[0])
        run.append(mk(20, 4))
        r2 = og.apply(*run[1])
        run.append(mk(700, 5))
        r3 = og.apply(*run[2])
        got = g.apply_many(run)
        assert [list(map(int, o)) for o in got] == [mod64(r1["F"]), mod64(r2["F"]), mod64(r3["F"])]
        step(40, 6, 1)
        g.set_tuning(local_max_pairs=0)
        step(20, 7, 0)
        step(600, 8, 0)
        g.set_tuning(local_max_pairs=50)
        step(25, 9, 1)
        assert g.count_static() == mod64(og.F)
        step(35, 10, 1)
        assert g.counts3() == oracle.static_counts3(og.row_ptr, og.col)


def test_all_eleven_types_follow_the_batches(gcb):
    """The six graphlets plus the five disconnected 4-vertex graphs, from the
    maintained counts, after region and edge-local batches; 128-bit values
    on a graph with millions of vertices."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    with gcb.Graph(n, rp, col, local_max_pairs=64) as g:
        assert g.counts_all() == oracle.counts_all(rp, col)
        for i, size in enumerate([30, 2000, 10]):
            ins, dels = gen.random_batch(n, gen.keys_from_csr(og.row_ptr, og.col), size // 2, size - size // 2, 70 + i)
            og.apply(ins, dels)
            g.apply(ins, dels)
            assert g.counts_all() == oracle.counts_all(og.row_ptr, og.col)
    big = 3_000_000
    edges = [(0, 1), (1, 2), (2, 0), (2, 3), (5, 6), (7, 8), (8, 9)]
    rp, col = csr_from_edges(big, edges)
    with gcb.Graph(big, rp, col) as g:
        got = g.counts_all()
        assert got == oracle.counts_all(rp, col)
        assert got[10] > (1 << 64) and sum(got) == __import__("math").comb(big, 4)
