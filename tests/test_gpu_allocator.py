"""Device memory through the gc_options allocator callbacks: PyTorch's
caching allocator behind every buffer of a handle.  The counts through a
stream of batches equal the oracle's, nothing stays allocated after
gc_close, and an allocation that fails makes the call return GC_ENOMEM with
the graph and its counts unchanged."""
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


def test_torch_allocator_carries_a_batch_stream(gcb):
    pytest.importorskip("torch")
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [1000, 10000, 1000, 10000], 0.5, 2)
    og = oracle.OracleGraph(rp, col)
    expect = [og.apply(i, d)["F"] for i, d in batches]
    alloc = gcb.TorchAllocator()
    with gcb.Graph(n, rp, col, allocator=alloc) as g:
        assert g.counts() == oracle.static_counts(rp, col)
        assert [g.apply(i, d) for i, d in batches] == expect
        assert g.count_static() == expect[-1]
        assert alloc.allocs > 0 and alloc.live
        # the library's own count of held bytes matches what the callbacks hold
        assert g.device_bytes() == sum(alloc.live.values())
    assert alloc.live == {}


def test_failed_allocation_leaves_the_graph_unchanged(gcb):
    pytest.importorskip("torch")
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    small, big = gen.batch_stream(n, keys, [100, 60000], 0.5, 12)
    alloc = gcb.TorchAllocator()
    with gcb.Graph(n, rp, col, allocator=alloc) as g:
        F1 = g.apply(*small)
        m1 = g.num_edges()
        alloc.fail = True
        # a batch far larger than any before needs larger batch scratch
        with pytest.raises(gcb.GCError) as ei:
            g.apply(*big)
        assert ei.value.code == gcb.GC_ENOMEM
        assert g.counts() == F1 and g.num_edges() == m1
        alloc.fail = False
        og = oracle.OracleGraph(*gen.csr_from_keys(n, gen.apply_batch_keys(keys, *small)))
        assert g.apply(*big) == og.apply(*big)["F"]
    assert alloc.live == {}


@pytest.mark.parametrize("after", [0, 3, 12])
def test_failed_open_returns_enomem_and_frees_what_it_took(gcb, after):
    """gc_open with the pool running dry after `after` allocations."""
    pytest.importorskip("torch")
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    alloc = gcb.TorchAllocator()
    alloc.fail_after = after
    with pytest.raises(gcb.GCError) as ei:
        gcb.Graph(n, rp, col, allocator=alloc)
    assert ei.value.code == gcb.GC_ENOMEM
    assert alloc.allocs == after
    assert alloc.live == {}
