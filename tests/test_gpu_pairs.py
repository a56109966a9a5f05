"""The two-batch form of sequential batched runs: when batch 0's region holds
most of the graph, the later batches go in pairs (the first committed without
a count, the second counted over every vertex, which gives the whole graph's
counts before and after it).  Every result must equal the oracle's Algorithm
2 steps and the plain form, through halts for pool space, with odd and even
run lengths, through the device API, and next to edge-local batches."""
import numpy as np
import pytest

import oracle
from gc_testutil import edges_from_csr
from synth import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gcb():
    from paper_2308_14493_gb300 import gc as binding

    binding.load()
    return binding


def _expect(rp, col, batches):
    og = oracle.OracleGraph(rp, col)
    return [og.apply(i, d)["F"] for i, d in batches], og


@pytest.mark.parametrize("k", [3, 4, 7])
def test_pairs_equal_the_oracle_and_the_single_pass_form(gcb, k):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [3000, 10000, 1000, 5000, 8000, 2000, 10000][:k], 0.5, 90 + k)
    expect, og = _expect(rp, col, batches)
    with gcb.Graph(n, rp, col) as g:
        assert g.apply_many(batches) == expect
        assert g.stats()["path"] == 2
        assert g.counts() == expect[-1] and g.count_static() == expect[-1]
        assert g.counts3() == oracle.static_counts3(og.row_ptr, og.col)
        got = g.export_csr()
        assert np.array_equal(got[0], og.row_ptr) and np.array_equal(got[1], og.col)
    with gcb.Graph(n, rp, col) as g:
        g.set_tuning(pair_min_share=0)
        assert g.apply_many(batches) == expect
        assert g.stats()["path"] == 0


def test_later_runs_pair_from_their_first_batch(gcb):
    """After a run whose first batch's region went in pairs, the handle
    keeps that batch's size: a later run whose first batch is at least as
    large pairs from batch 0 (four batches: two pairs, no batch alone),
    with the same counts; a smaller first batch measures its region again;
    setting the tuning forgets the size."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    stream = gen.batch_stream(n, keys, [5000, 4000, 3000, 8000, 6000, 7000, 5000, 500, 6000, 6000, 6000],
                              0.5, 97)
    runs = [stream[0:3], stream[3:7], stream[7:10], stream[10:11]]
    expect, _ = _expect(rp, col, stream)
    with gcb.Graph(n, rp, col) as g:
        at = 0
        launches, paths = [], []
        for run in runs:
            assert g.apply_many(run) == expect[at:at + len(run)]
            launches.append(g.stats()["launches"])
            paths.append(g.stats()["path"])
            at += len(run)
        assert paths[:2] == [2, 2]
        assert g.counts() == expect[-1] and g.count_static() == expect[-1]
    # the second run (first batch 8,000 >= 5,000) took two passes for four
    # batches; the same four batches from a fresh handle take three
    with gcb.Graph(n, rp, col) as g:
        assert g.apply_many(stream[0:3]) == expect[0:3]
        g.set_tuning(**g.tuning())
        assert g.apply_many(stream[3:7]) == expect[3:7]
        assert g.stats()["launches"] > launches[1]


def test_small_regions_do_not_pair(gcb):
    """Batches of a few pairs on a sparse graph: batch 0's region is a small
    part of the graph, so the run stays one pass per batch."""
    n = 20000
    keys = gen.er_graph(n, 30000, 5)
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [3, 4, 5, 6], 0.5, 6, ins_weighting="uniform")
    expect, _ = _expect(rp, col, batches)
    with gcb.Graph(n, rp, col) as g:
        assert g.apply_many(batches) == expect
        assert g.stats()["path"] == 0


def test_pairs_through_halts_for_pool_space(gcb):
    """Insertions into many nearly full hub rows: commits of both kinds of
    batch in a pair run out of pool space, the run halts, the host grows the
    pool and finishes the pending commit, and the pairs resume."""
    n = 3000
    rng = np.random.default_rng(31)
    keys = set(int(x) for x in gen.er_graph(n, 3000, 30))
    hubs = list(range(20))
    for h in hubs:
        for v in rng.choice(np.arange(20, n), 500, replace=False):
            keys.add((h << 32) | int(v))
    keys = np.array(sorted(keys), dtype=np.uint64)
    rp, col = gen.csr_from_keys(n, keys)
    og = oracle.OracleGraph(rp, col)
    batches, expect = [], []
    for _ in range(7):
        cur = set(int(x) for x in gen.keys_from_csr(og.row_ptr, og.col))
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
    with gcb.Graph(n, rp, col, slack=0.05) as g:
        g.set_tuning(pair_min_share=1)
        assert g.apply_many(batches) == expect
        st = g.stats()
        assert st["path"] == 2 and st["relayouts"] >= 2
        got = g.export_csr()
        assert np.array_equal(got[0], og.row_ptr) and np.array_equal(got[1], og.col)


def test_device_runs_pair_and_a_bad_pair_turns_pairing_off(gcb):
    torch = pytest.importorskip("torch")
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [4000, 6000, 2000, 9000, 3000], 0.5, 71)
    pairs, desc, off = [], [], 0
    for ins, dels in batches:
        desc.append((off, len(ins), off + len(ins), len(dels)))
        pairs += [ins, dels]
        off += len(ins) + len(dels)
    flat = np.ascontiguousarray(np.concatenate(pairs).astype(np.int32))
    d_pairs = torch.from_numpy(flat).cuda()
    torch.cuda.synchronize()
    expect, _ = _expect(rp, col, batches)
    with gcb.Graph(n, rp, col) as g:
        assert gcb.gc_apply_batches_device(g.h, d_pairs.data_ptr(), desc) == expect
        assert g.stats()["path"] == 2
    # a self-loop in batch 3: the run does not pair, and that batch is not applied
    bad = flat.copy()
    bad[desc[3][0]] = (bad[desc[3][0]][0], bad[desc[3][0]][0])
    d_bad = torch.from_numpy(bad).cuda()
    torch.cuda.synchronize()
    with gcb.Graph(n, rp, col) as g1, gcb.Graph(n, rp, col) as g2:
        g2.set_tuning(pair_min_share=0)
        try:
            r1 = gcb.gc_apply_batches_device(g1.h, d_bad.data_ptr(), desc)
        except gcb.GCError as e:
            r1 = e.code
        assert g1.stats()["path"] == 0
        try:
            r2 = gcb.gc_apply_batches_device(g2.h, d_bad.data_ptr(), desc)
        except gcb.GCError as e:
            r2 = e.code
        assert r1 == r2 and g1.counts() == g2.counts()


def test_pairs_next_to_edge_local_batches(gcb):
    """A run mixing region batches (paired) with small batches that take the
    edge-local delta: the local form must not use triangle sums the unpaired
    commits left stale."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    sizes = [5000, 4000, 6000, 20, 30, 5000, 7000, 3000, 40]
    batches = gen.batch_stream(n, keys, sizes, 0.5, 123)
    expect, _ = _expect(rp, col, batches)
    with gcb.Graph(n, rp, col, local_max_pairs=64) as g:
        assert g.apply_many(batches) == expect
        assert g.count_static() == expect[-1]
        # and plain local batches afterwards
        n2, k2 = n, gen.apply_batch_keys(keys, *batches[0])
        for ins, dels in batches[1:]:
            k2 = gen.apply_batch_keys(k2, ins, dels)
        more = gen.batch_stream(n2, k2, [10, 25, 50], 0.5, 124)
        og = oracle.OracleGraph(*gen.csr_from_keys(n2, k2))
        for ins, dels in more:
            assert g.apply(ins, dels) == og.apply(ins, dels)["F"]
            assert g.stats()["path"] == 1


def _dirty(rng, n, keys, base_ins, base_dels, shared):
    """A raw batch with repeats, a pair in both A and D, a no-op insertion
    (an existing edge) and a no-op deletion (an absent pair), plus `shared`
    pairs that another batch of the run also carries."""
    ins = [tuple(x) for x in base_ins] + [tuple(base_ins[0][::-1])] + [tuple(x) for x in shared]
    dels = [tuple(x) for x in base_dels] + [tuple(base_dels[0])]
    both = base_ins[1]
    dels.append(tuple(both))
    e = int(keys[rng.integers(len(keys))])
    ins.append((e >> 32, e & 0xFFFFFFFF))
    while True:
        a, b = (int(x) for x in rng.integers(0, n, 2))
        kk = (min(a, b) << 32) | max(a, b)
        if a != b and not np.any(keys == kk):
            dels.append((a, b))
            break
    return np.array(ins, np.int32), np.array(dels, np.int32)


@pytest.mark.parametrize("k", [3, 4, 7])
def test_twin_passes_of_independent_batches(gcb, k):
    """Independent batches on one snapshot: batch 0 alone, then two batches
    per pass (each with its own batch tag in the normalisation keys).  Every
    result is the oracle's Algorithm 2 step on the snapshot, and the graph
    and its counts stay as they were."""
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    rng = np.random.default_rng(200 + k)
    base = gen.batch_stream(n, keys, [2000, 5000, 800, 9000, 3000, 1500, 6000][:k], 0.5, 210 + k,
                            sequential=False)
    shared = [tuple(base[0][0][j]) for j in range(5)] + [tuple(base[0][1][0])]
    batches = [_dirty(rng, n, keys, i, d, shared if b % 2 else shared[:2]) for b, (i, d) in enumerate(base)]
    F0 = oracle.static_counts(rp, col)
    expect = [oracle.fdgc_step(rp, col, i, d, F0)["F"] for i, d in batches]
    with gcb.Graph(n, rp, col) as g:
        assert g.apply_many(batches, independent=True) == expect
        assert g.stats()["path"] == 2
        assert g.counts() == F0 and g.num_edges() == len(keys)
        assert g.count_static() == F0
    with gcb.Graph(n, rp, col) as g:
        g.set_tuning(pair_min_share=0)
        assert g.apply_many(batches, independent=True) == expect
        assert g.stats()["path"] == 0


def test_twin_passes_through_the_device_api_and_local_batches(gcb):
    torch = pytest.importorskip("torch")
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    sizes = [3000, 12, 7000, 40, 5000, 4000, 9, 6000]
    batches = gen.batch_stream(n, keys, sizes, 0.5, 77, sequential=False)
    F0 = oracle.static_counts(rp, col)
    expect = [oracle.fdgc_step(rp, col, i, d, F0)["F"] for i, d in batches]
    pairs, desc, off = [], [], 0
    for ins, dels in batches:
        desc.append((off, len(ins), off + len(ins), len(dels)))
        pairs += [ins, dels]
        off += len(ins) + len(dels)
    d_pairs = torch.from_numpy(np.ascontiguousarray(np.concatenate(pairs).astype(np.int32))).cuda()
    torch.cuda.synchronize()
    for local in (0, 64):
        with gcb.Graph(n, rp, col, local_max_pairs=local) as g:
            assert gcb.gc_apply_batches_device(g.h, d_pairs.data_ptr(), desc, independent=True) == expect
            assert g.counts() == F0
