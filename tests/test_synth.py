"""The seeded input generators (synth/gen.py) that both the oracle tests and
the GPU path draw from: the counter-based generator against the published
splitmix64 outputs, and the graphs and batches against the recipe (exact
sizes, no loops or repeats, deletions of present edges, insertions of
absent pairs, reproducible from the seed).  CPU only."""
import numpy as np

from synth import gen


def test_splitmix64_matches_its_published_outputs():
    # the first outputs of splitmix64 started from state 0
    got = gen.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = gen.uniform01(7, 0, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def _check_simple(n, keys, m):
    keys = np.asarray(keys, dtype=np.uint64)
    assert keys.size == m
    assert np.all(np.diff(keys.astype(np.float64)) > 0) or m < 2        # sorted, distinct
    u = (keys >> np.uint64(32)).astype(np.int64)
    v = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert np.all(u < v) and np.all(v < n)                               # canonical, no loops


def test_graphs_have_exact_sizes_and_are_reproducible():
    n, keys = gen.workload_graph("c1")
    _check_simple(n, keys, 20000)
    n2, keys2 = gen.workload_graph("c2")
    _check_simple(n2, keys2, 100000)
    assert np.array_equal(keys2, gen.workload_graph("c2")[1])
    cl = gen.chung_lu_graph(5000, 40000, 2.1, 400.0, 3)
    _check_simple(5000, cl, 40000)
    assert not np.array_equal(cl, gen.chung_lu_graph(5000, 40000, 2.1, 400.0, 4))
    deg = np.diff(gen.csr_from_keys(5000, cl)[0])
    assert deg.max() <= 400 * 1.5 and deg.max() > 8 * deg.mean()         # capped, heavy-tailed


def test_csr_round_trip_is_symmetric_and_sorted():
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    assert rp[-1] == 2 * keys.size
    for x in range(0, n, 97):
        row = col[rp[x]:rp[x + 1]]
        assert np.all(np.diff(row) > 0)
        for y in row[:5]:
            assert x in col[rp[y]:rp[y + 1]]
    assert np.array_equal(gen.keys_from_csr(rp, col), keys)


def test_batches_follow_the_recipe():
    n, keys = gen.workload_graph("c2")
    present = set(int(k) for k in keys)
    for weighting in ("degree", "uniform"):
        ins, dels = gen.random_batch(n, keys, 300, 200, 5, ins_weighting=weighting)
        assert ins.shape == (300, 2) and dels.shape == (200, 2)
        ik = [(min(a, b) << 32) | max(a, b) for a, b in ins.tolist()]
        dk = [(min(a, b) << 32) | max(a, b) for a, b in dels.tolist()]
        assert len(set(ik)) == 300 and len(set(dk)) == 200
        assert all(k not in present for k in ik) and all(k in present for k in dk)
        assert all(a != b for a, b in ins.tolist())
    a1, d1 = gen.random_batch(n, keys, 50, 50, 9)
    a2, d2 = gen.random_batch(n, keys, 50, 50, 9)
    assert np.array_equal(a1, a2) and np.array_equal(d1, d2)


def test_sequential_stream_is_valid_against_the_evolving_graph():
    n, keys = gen.workload_graph("c1")
    cur = set(int(k) for k in keys)
    for ins, dels in gen.batch_stream(n, keys, [100, 40, 300], 0.6, 2):
        ik = {(min(a, b) << 32) | max(a, b) for a, b in ins.tolist()}
        dk = {(min(a, b) << 32) | max(a, b) for a, b in dels.tolist()}
        assert not (ik & cur) and dk <= cur
        cur = (cur - dk) | ik
