"""Serving (request loop over resident graphs): every result equals the same
batch applied alone, in order, to a fresh copy of its graph; requests of
different graphs overlap; admission by device memory releases idle scratch
and still gives the same results."""
import threading
import time

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


def _graphs():
    specs = [gen.WORKLOADS["c1"], gen.WORKLOADS["c2"],
             dict(kind="cl", n=20000, m=150000, gamma=2.2, dmax=800.0, seed=5),
             dict(kind="er", n=3000, m=9000, seed=6)]
    out = []
    for p in specs:
        n, keys = gen.workload_graph(p)
        out.append((n, keys))
    return out


def _requests(graphs, count, seed):
    """A seeded mix: per graph a sequential stream; the interleaving is
    seeded too.  Returns [(graph, ins, dels)] in submission order."""
    rng = np.random.default_rng(seed)
    per = [[] for _ in graphs]
    counts = np.bincount(rng.integers(0, len(graphs), count), minlength=len(graphs))
    for gi, (n, keys) in enumerate(graphs):
        sizes = [int(x) for x in np.exp(rng.uniform(np.log(5), np.log(3000), counts[gi]))]
        per[gi] = gen.batch_stream(n, keys, sizes, 0.7, 100 + gi) if sizes else []
    order = np.concatenate([np.full(c, gi) for gi, c in enumerate(counts)])
    rng.shuffle(order)
    cursor = [0] * len(graphs)
    out = []
    for gi in order:
        ins, dels = per[gi][cursor[gi]]
        cursor[gi] += 1
        out.append((int(gi), ins, dels))
    return out


def _alone(gcb, graphs, reqs):
    """Each graph's requests applied in order on a fresh handle, one at a time."""
    res = {}
    handles = [gcb.Graph(n, *gen.csr_from_keys(n, keys)) for n, keys in graphs]
    for i, (gi, ins, dels) in enumerate(reqs):
        res[i] = handles[gi].apply(ins, dels)
    for h in handles:
        h.close()
    return res


def _served(gcb, graphs, reqs, slots, budget=0, spacing_s=0.0):
    handles = [gcb.Graph(n, *gen.csr_from_keys(n, keys)) for n, keys in graphs]
    results = {}
    with gcb.Server(handles, slots=slots, hbm_budget_bytes=budget) as srv:
        tickets = []

        def submit():
            for gi, ins, dels in reqs:
                tickets.append(srv.submit(gi, ins, dels))
                if spacing_s:
                    time.sleep(spacing_s)

        t = threading.Thread(target=submit)
        t.start()
        t.join()
        for i, tk in enumerate(tickets):
            results[i] = srv.wait(tk)
        counters = srv.counters()
    finals = [h.counts() for h in handles]
    edges = [h.num_edges() for h in handles]
    for h in handles:
        h.close()
    return results, counters, finals, edges


def test_served_mix_equals_alone(gcb):
    graphs = _graphs()
    reqs = _requests(graphs, 48, 7)
    alone = _alone(gcb, graphs, reqs)
    served, (peak, _), _, _ = _served(gcb, graphs, reqs, slots=4)
    for i in range(len(reqs)):
        r = served[i]
        assert r["status"] == 0
        assert r["graph"] == reqs[i][0]
        assert r["counts"] == alone[i], f"request {i} on graph {reqs[i][0]}"
        assert r["t_submit_ms"] <= r["t_admit_ms"] <= r["t_done_ms"]
    # the loop ran requests of different graphs at the same time
    assert peak >= 2


def test_served_results_match_oracle_on_a_small_graph(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    batches = gen.batch_stream(n, keys, [50, 400, 7, 1200], 0.7, 11)
    og = oracle.OracleGraph(rp, col)
    expect = [og.apply(i, d)["F"] for i, d in batches]
    with gcb.Graph(n, rp, col) as g:
        with gcb.Server([g], slots=2) as srv:
            tickets = [srv.submit(0, i, d) for i, d in batches]
            got = [srv.wait(t)["counts"] for t in tickets]
        assert got == expect
        assert g.counts() == expect[-1]


def test_admission_under_a_tight_budget_gives_same_results(gcb):
    graphs = _graphs()
    reqs = _requests(graphs, 24, 8)
    alone = _alone(gcb, graphs, reqs)
    # a budget barely above what the open graphs hold: idle scratch must be
    # released and requests wait for running ones
    handles = [gcb.Graph(n, *gen.csr_from_keys(n, keys)) for n, keys in graphs]
    held = sum(h.device_bytes() for h in handles)
    for h in handles:
        h.close()
    served, (peak, trims), _, _ = _served(gcb, graphs, reqs, slots=4, budget=held + (256 << 10))
    for i in range(len(reqs)):
        assert served[i]["status"] == 0
        assert served[i]["counts"] == alone[i]
    # the first batch on a graph grows its scratch; later ones may fit in it
    assert any(served[i]["bytes_predicted"] > 0 for i in range(len(reqs)))
    assert trims >= 1


def test_batch_bytes_and_trim(gcb):
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    ins, dels = gen.random_batch(n, keys, 3000, 2000, 12)
    with gcb.Graph(n, rp, col) as g:
        before = g.device_bytes()
        pred = gcb.gc_batch_bytes(g.h, 3000, 2000)
        assert pred > 0
        out = g.apply(ins, dels)
        grown = g.device_bytes() - before
        assert 0 <= grown <= pred
        g.trim()
        assert g.device_bytes() < before + grown
        # the next batch re-creates the scratch and still counts right
        ins2, dels2 = gen.random_batch(n, keys, 100, 100, 13)
        og = oracle.OracleGraph(rp, col)
        assert out == og.apply(ins, dels)["F"]
        assert g.apply(ins2, dels2) == og.apply(ins2, dels2)["F"]


def test_submit_errors(gcb):
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    with gcb.Graph(n, rp, col) as g:
        with gcb.Server([g], slots=1) as srv:
            with pytest.raises(gcb.GCError):
                srv.submit(1, [[0, 1]], None)
            with pytest.raises(gcb.GCError):
                srv.wait(12345)
            # a batch with a bad id fails alone and changes nothing
            bad = srv.submit(0, [[0, n]], None)
            r = srv.wait(bad)
            assert r["status"] != 0
            ok = srv.submit(0, None, None)
            assert srv.wait(ok)["status"] == 0
        assert g.counts() == oracle.static_counts(rp, col)
