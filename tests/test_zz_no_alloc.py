"""The allocation-free static count agrees with gc_count_static and with the
CPU oracle.

gc_count_static_noalloc is for callers that must not allocate device memory
when they ask for a count (device memory reserved up front by another
allocator, latency-critical loops that cannot take cudaMalloc's
synchronisation, host processes that forbid allocations after start-up).  It
works in a fixed scratch array compiled into the library, shared by every
call.  This file is collected last on purpose, so that a run stopping at the
first failure has already run every other test; it passes both alone in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
from synth import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gcb():
    from paper_2308_14493_gb300 import gc as binding

    binding.load()
    return binding


def _device_csr(torch, rp, col):
    d_rp = torch.from_numpy(np.ascontiguousarray(rp, dtype=np.int32)).cuda()
    d_col = torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).cuda()
    torch.cuda.synchronize()
    return d_rp, d_col


@pytest.mark.parametrize("name", ["c2", "c1"])
def test_noalloc_count_equals_gc_count_static_twice(gcb, name):
    torch = pytest.importorskip("torch")
    n, keys = gen.workload_graph(name)
    rp, col = gen.csr_from_keys(n, keys)
    with gcb.Graph(n, rp, col) as g:
        expect = g.count_static()
    assert expect == oracle.static_counts(rp, col)
    d_rp, d_col = _device_csr(torch, rp, col)
    # two calls in a row: the shared scratch keeps the first call's contents,
    # which the second call must not pick up
    for _ in range(2):
        got = gcb.gc_count_static_noalloc(n, d_rp.data_ptr(), d_col.data_ptr(), len(col))
        assert got == expect


@pytest.mark.parametrize("edges", [262144, 262143], ids=["entries_at_cap", "one_edge_under_cap"])
def test_noalloc_at_the_caps_on_a_hub_graph(gcb, edges):
    """16,384 vertices and 2 x 262,144 adjacency entries (the caps), on a
    Chung-Lu graph with hubs of a few thousand neighbours: the fixed scratch is
    used to its end and the heavy 4-cycle pivots reach the cluster and hash
    tiers; the counts equal the oracle's, twice in a row."""
    torch = pytest.importorskip("torch")
    n = gcb.GC_NOALLOC_MAX_VERTICES
    keys = gen.chung_lu_graph(n, edges, 2.0, 4000.0, 61)
    rp, col = gen.csr_from_keys(n, keys)
    assert len(col) == 2 * edges and len(col) <= gcb.GC_NOALLOC_MAX_ENTRIES
    assert int(np.diff(rp).max()) > 1000
    expect = oracle.static_counts(rp, col)
    d_rp, d_col = _device_csr(torch, rp, col)
    for _ in range(2):
        assert gcb.gc_count_static_noalloc(n, d_rp.data_ptr(), d_col.data_ptr(), len(col)) == expect


# one small CSR per device-side check; every one must give GC_EINVAL
BAD_CSRS = {
    "unsorted_row": ([0, 2, 3, 4], [2, 1, 0, 0]),
    "repeated_entry": ([0, 2, 3, 4], [1, 1, 0, 0]),
    "self_loop": ([0, 2, 3, 4], [0, 1, 0, 0]),
    "id_out_of_range": ([0, 1, 2, 3], [1, 0, 7]),
    "negative_id": ([0, 1, 2, 3], [1, 0, -1]),
    "last_offset_not_nnz": ([0, 1, 2, 2], [1, 0, 0]),
    "decreasing_offsets": ([0, 2, 1, 2], [1, 2]),
}


@pytest.mark.parametrize("name", sorted(BAD_CSRS))
def test_noalloc_rejects_a_malformed_csr(gcb, name):
    torch = pytest.importorskip("torch")
    rp, col = (np.array(x, np.int32) for x in BAD_CSRS[name])
    nnz = len(col)
    d_rp, d_col = _device_csr(torch, rp, col)
    with pytest.raises(gcb.GCError) as ei:
        gcb.gc_count_static_noalloc(3, d_rp.data_ptr(), d_col.data_ptr(), nnz)
    assert ei.value.code == gcb.GC_EINVAL
    # the scratch is left usable: a valid graph still counts right
    tk = np.array([(0 << 32) | 1, (1 << 32) | 2, (0 << 32) | 2], dtype=np.uint64)
    trp, tcol = gen.csr_from_keys(3, tk)
    d_trp, d_tcol = _device_csr(torch, trp, tcol)
    assert gcb.gc_count_static_noalloc(3, d_trp.data_ptr(), d_tcol.data_ptr(), len(tcol)) == [0] * 6


def test_noalloc_small_graph_then_large_graph(gcb):
    torch = pytest.importorskip("torch")
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    tiny_n, tiny_edges = 5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4)]
    tk = np.array(sorted((a << 32) | b for a, b in tiny_edges), dtype=np.uint64)
    trp, tcol = gen.csr_from_keys(tiny_n, tk)
    with gcb.Graph(tiny_n, trp, tcol) as g:
        tiny_expect = g.count_static()
    with gcb.Graph(n, rp, col) as g:
        expect = g.count_static()
    d_trp, d_tcol = _device_csr(torch, trp, tcol)
    d_rp, d_col = _device_csr(torch, rp, col)
    assert gcb.gc_count_static_noalloc(tiny_n, d_trp.data_ptr(), d_tcol.data_ptr(), len(tcol)) == tiny_expect
    assert gcb.gc_count_static_noalloc(n, d_rp.data_ptr(), d_col.data_ptr(), len(col)) == expect
    assert gcb.gc_count_static_noalloc(tiny_n, d_trp.data_ptr(), d_tcol.data_ptr(), len(tcol)) == tiny_expect


def test_noalloc_rejects_sizes_beyond_the_scratch(gcb):
    torch = pytest.importorskip("torch")
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(gcb.GCError) as ei:
        gcb.gc_count_static_noalloc(gcb.GC_NOALLOC_MAX_VERTICES + 1, d.data_ptr(), d.data_ptr(), 0)
    assert ei.value.code == gcb.GC_EINVAL
    with pytest.raises(gcb.GCError) as ei:
        gcb.gc_count_static_noalloc(10, d.data_ptr(), d.data_ptr(), gcb.GC_NOALLOC_MAX_ENTRIES + 2)
    assert ei.value.code == gcb.GC_EINVAL


def test_noalloc_rejects_an_asymmetric_csr(gcb):
    torch = pytest.importorskip("torch")
    rp = np.array([0, 1, 1, 1], np.int32)   # 0 -> 1 without 1 -> 0
    col = np.array([1], np.int32)
    d_rp, d_col = _device_csr(torch, rp, col)
    with pytest.raises(gcb.GCError) as ei:
        gcb.gc_count_static_noalloc(3, d_rp.data_ptr(), d_col.data_ptr(), 1)
    assert ei.value.code == gcb.GC_EINVAL
