"""A seeded random program of every kind of call on one handle, checked
against the oracle after each step: plain batches of every size (region and
edge-local forms), what-if batches, batched runs (sequential and
independent), vertex deletions and insertions, tuning changes and static
recounts.  Counts must stay bit-exact throughout, and (in two of the
programs) the per-vertex and per-edge orbit counts of the final graph must
equal the oracle's."""
import numpy as np
import pytest

import oracle
from synth import gen
from gc_testutil import csr_from_edges, edges_from_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gcb():
    from paper_2308_14493_gb300 import gc as binding

    binding.load()
    return binding


def mod64(xs):
    return [int(x) & 0xFFFFFFFFFFFFFFFF for x in xs]


def _batch(rng, n, rp, col, size):
    keys = gen.keys_from_csr(rp, col)
    k_ins = int(rng.integers(0, size + 1))
    ins, dels = gen.random_batch(n, keys, k_ins, size - k_ins, int(rng.integers(1 << 30)))
    return ins, dels


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_random_program_of_calls(gcb, seed):
    rng = np.random.default_rng(seed)
    n0 = 1500
    keys = gen.chung_lu_graph(n0, 12000, 2.1, 300.0, seed)
    rp, col = gen.csr_from_keys(n0, keys)
    og = oracle.OracleGraph(rp, col)
    n = n0
    with gcb.Graph(n, rp, col, local_max_pairs=int(rng.choice([0, 16, 64, 256]))) as g:
        for step in range(60):
            op = rng.choice(["apply", "apply", "apply", "whatif", "run", "indep", "delv", "addv", "tune", "recount"])
            if op == "apply":
                ins, dels = _batch(rng, n, og.row_ptr, og.col, int(rng.choice([1, 5, 30, 120, 600, 2500])))
                r = og.apply(ins, dels)
                assert g.apply(ins, dels) == mod64(r["F"]), (step, op)
            elif op == "whatif":
                ins, dels = _batch(rng, n, og.row_ptr, og.col, int(rng.choice([3, 40, 900])))
                r = oracle.fdgc_step(og.row_ptr, og.col, ins, dels, og.F, 3)
                assert g.count_batch(ins, dels) == mod64(r["F"]), (step, op)
            elif op == "run":
                batches = [_batch(rng, n, og.row_ptr, og.col, int(rng.choice([2, 50, 700]))) for _ in range(4)]
                expect = [mod64(og.apply(i, d)["F"]) for i, d in batches]
                got = g.apply_many(batches)
                assert [list(map(int, o)) for o in got] == expect, (step, op)
            elif op == "indep":
                batches = [_batch(rng, n, og.row_ptr, og.col, int(rng.choice([2, 50, 700]))) for _ in range(4)]
                expect = [mod64(oracle.fdgc_step(og.row_ptr, og.col, i, d, og.F, 3)["F"]) for i, d in batches]
                got = g.apply_many(batches, independent=True)
                assert [list(map(int, o)) for o in got] == expect, (step, op)
            elif op == "delv":
                ids = [int(x) for x in rng.integers(0, n, size=int(rng.integers(1, 4)))]
                drop = set(ids)
                kept = [(u, v) for u, v in edges_from_csr(og.row_ptr, og.col) if u not in drop and v not in drop]
                rp2, col2 = csr_from_edges(n, kept)
                og = oracle.OracleGraph(rp2, col2)
                assert g.delete_vertices(ids) == mod64(og.F), (step, op)
            elif op == "addv":
                k = int(rng.integers(1, 20))
                assert g.add_vertices(k) == n
                n += k
                rp2 = np.concatenate([og.row_ptr, np.full(k, og.row_ptr[-1], np.int64)])
                og = oracle.OracleGraph(rp2, og.col)
                # join a few of them at once
                ins = np.array([(n - 1 - j, int(rng.integers(0, n - k))) for j in range(min(k, 5))], np.int32)
                r = og.apply(ins, np.zeros((0, 2), np.int32))
                assert g.apply(ins, None) == mod64(r["F"]), (step, op)
            elif op == "tune":
                g.set_tuning(local_max_pairs=int(rng.choice([0, 8, 100, 1000])))
            else:
                assert g.count_static() == mod64(og.F), (step, op)
            assert g.counts() == mod64(og.F), (step, op)
        assert g.counts3() == oracle.static_counts3(og.row_ptr, og.col)
        assert g.counts_all() == oracle.counts_all(og.row_ptr, og.col)
        grp, gcol = g.export_csr()
        assert np.array_equal(grp.astype(np.int64), og.row_ptr) and np.array_equal(gcol, og.col)
        if seed > 2:   # the oracle's local counts take seconds: two programs check them
            return
        # local counts of the final graph (new vertices and relocated rows included)
        assert g.vertex_orbits().astype(np.int64).tolist() == oracle.vertex_orbits(og.row_ptr, og.col)
        edges, orb = g.edge_orbits()
        keys, rows = oracle.edge_orbits(og.row_ptr, og.col)
        assert edges.tolist() == [list(k) for k in keys]
        assert orb.astype(np.int64).tolist() == rows
