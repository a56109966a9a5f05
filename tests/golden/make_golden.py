"""Write oracle results on the seeded workloads.

Calls only the CPU oracle (``oracle/``) and the seeded generators (``synth``).
Run from the repository root:

    python tests/golden/make_golden.py           # workloads.json (seconds)
    python tests/golden/make_golden.py --large   # workloads_large.json (tens of minutes)
    python tests/golden/make_golden.py --large c3_local   # one part of it, merged in (also c3_local_10k)
    python tests/golden/make_golden.py --c5 g0   # workloads_c5.json, one part (g0, g7, g0_stream)

Each part runs alone and is merged into its file, so parts can run as
separate processes.
"""
import fcntl
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from synth import gen  # noqa: E402


def main():
    out = {}
    # ER n=2,000 m=20,000 (seed 0); one batch of 200 deletions of existing
    # edges + 200 insertions of uniform non-edges (seed 1)
    n, keys = gen.workload_graph("c1")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col, "literal")
    ins, dels = gen.random_batch(n, keys, 200, 200, 1, ins_weighting="uniform")
    r = oracle.fdgc_step(rp, col, ins, dels, F0, 3, "literal")
    out["c1"] = dict(static=F0, after=r["F"], Ca=r["Ca"], Cb=r["Cb"], sums_a=r["sums_a"], sums_b=r["sums_b"],
                     region_vertices=r["region_vertices"], edges_a=r["edges_a"], edges_b=r["edges_b"])
    # Chung-Lu n=7,000 m=100,000 gamma 2.1 dmax 1,000 (seed 0); sequential
    # 50/50 batches of 1,000 and 10,000 (seed 2)
    n, keys = gen.workload_graph("c2")
    rp, col = gen.csr_from_keys(n, keys)
    g = oracle.OracleGraph(rp, col)
    steps = [dict(static=list(g.F))]
    for ins, dels in gen.batch_stream(n, keys, [1000, 10000], 0.5, 2):
        r = g.apply(ins, dels)
        steps.append(dict(after=r["F"], Ca=r["Ca"], Cb=r["Cb"], region_vertices=r["region_vertices"]))
    out["c2"] = steps
    with open(os.path.join(HERE, "workloads.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


def _merge(name, part):
    """Merge ``part`` (a dict) into the JSON file ``name`` beside this script."""
    path = os.path.join(HERE, name)
    fd = os.open(HERE, os.O_RDONLY)
    try:
        fcntl.flock(fd, fcntl.LOCK_EX)   # parts may finish at the same time
        out = {}
        if os.path.exists(path):
            with open(path) as f:
                out = json.load(f)
        out.update(part)
        with open(path + ".tmp", "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        os.replace(path + ".tmp", path)
    finally:
        os.close(fd)


def large_c3_local():
    """The c3 graph after the sequential stream of small 70/30 batches (sizes
    10, 100, 1,000, 10, 100; batch seed 77) that the edge-local test applies:
    the oracle's static count of the final edge set, which the maintained
    counts must equal."""
    n, keys = gen.workload_graph("c3")
    sizes = [10, 100, 1000, 10, 100]
    cur = keys
    for ins, dels in gen.batch_stream(n, keys, sizes, 0.7, 77):
        cur = gen.apply_batch_keys(cur, ins, dels)
    rp, col = gen.csr_from_keys(n, cur)
    return {"c3_local_stream": dict(sizes=sizes, seed=77, edges=int(cur.size), final=oracle.static_counts(rp, col))}


def large_c3_local_10k():
    """The c3 graph after one 10,000-update batch (70% insertions, batch seed
    78), the size at which the edge-local delta still beats the region
    recount there: the oracle's static count of the final edge set."""
    n, keys = gen.workload_graph("c3")
    ins, dels = gen.batch_stream(n, keys, [10000], 0.7, 78)[0]
    cur = gen.apply_batch_keys(keys, ins, dels)
    rp, col = gen.csr_from_keys(n, cur)
    return {"c3_local_10k": dict(size=10000, seed=78, edges=int(cur.size), final=oracle.static_counts(rp, col))}


def c5_graph(gi):
    """One graph of the serving workload: its static count and one
    100,000-update batch (70% insertions, batch seed 500 + gi) applied by the
    oracle's Algorithm 2 step."""
    p = gen.c5_graph_params()[gi]
    n, keys = gen.workload_graph(p)
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    ins, dels = gen.batch_stream(n, keys, [100000], 0.7, 500 + gi)[0]
    r = oracle.fdgc_step(rp, col, ins, dels, F0, 3)
    return {f"g{gi}": dict(params=p, static=F0, after=r["F"], Ca=r["Ca"], Cb=r["Cb"],
                           region_vertices=r["region_vertices"], n_ins=r["n_ins"], n_del=r["n_del"])}


def c5_stream(gi):
    """A sequential stream of 5 batches on one serving graph: sizes
    log-uniform in [100, 100,000] (seed 5), 70% insertions, batch seed
    510 + gi; the counts after every batch."""
    p = gen.c5_graph_params()[gi]
    n, keys = gen.workload_graph(p)
    rp, col = gen.csr_from_keys(n, keys)
    sizes = gen.log_uniform_sizes(5, 100, 100000, 5)
    og = oracle.OracleGraph(rp, col)
    steps = [dict(static=list(og.F))]
    for ins, dels in gen.batch_stream(n, keys, sizes, 0.7, 510 + gi):
        r = og.apply(ins, dels)
        steps.append(dict(after=r["F"], n_ins=r["n_ins"], n_del=r["n_del"]))
    return {f"g{gi}_stream": dict(sizes=sizes, seed=510 + gi, steps=steps)}


def main_large():
    """Full-size graphs: static counts and the first batch of each stream."""
    out = {}
    # Chung-Lu n=1.6M m=30M gamma 2.3 dmax 10,000; batches of 100,000
    # (60% insertions, 40% deletions), batch seed 3
    n, keys = gen.workload_graph("c3")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    ins, dels = gen.batch_stream(n, keys, [100000], 0.6, 3)[0]
    r = oracle.fdgc_step(rp, col, ins, dels, F0, 3)
    out["c3"] = dict(static=F0, after=r["F"], Ca=r["Ca"], Cb=r["Cb"], region_vertices=r["region_vertices"],
                     n_ins=r["n_ins"], n_del=r["n_del"])
    # Chung-Lu n=2.4M m=5M gamma 1.8 dmax 100,000; independent 50/50 batches
    # of log-uniform size in [10, 50,000], batch seed 4
    n, keys = gen.workload_graph("c4")
    rp, col = gen.csr_from_keys(n, keys)
    F0 = oracle.static_counts(rp, col)
    sizes = gen.log_uniform_sizes(64, 10, 50000, 4)
    batches = gen.batch_stream(n, keys, sizes[:3], 0.5, 4, sequential=False)
    res = []
    for ins, dels in batches:
        r = oracle.fdgc_step(rp, col, ins, dels, F0, 3)
        res.append(dict(after=r["F"], Ca=r["Ca"], Cb=r["Cb"], region_vertices=r["region_vertices"]))
    out["c4"] = dict(static=F0, sizes=sizes[:3], batches=res)
    _merge("workloads_large.json", out)


if __name__ == "__main__":
    if "--c5" in sys.argv:
        parts = sys.argv[sys.argv.index("--c5") + 1:] or ["g0", "g7", "g0_stream"]
        for part in parts:
            res = c5_stream(int(part[1:-7])) if part.endswith("_stream") else c5_graph(int(part[1:]))
            _merge("workloads_c5.json", res)
    elif "--large" in sys.argv and sys.argv[-1] == "c3_local":
        _merge("workloads_large.json", large_c3_local())
    elif "--large" in sys.argv and sys.argv[-1] == "c3_local_10k":
        _merge("workloads_large.json", large_c3_local_10k())
    elif "--large" in sys.argv:
        main_large()
    else:
        main()
