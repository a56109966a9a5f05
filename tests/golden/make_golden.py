"""Write oracle results on the seeded workloads.

Calls only the CPU oracle (``oracle/``) and the seeded generators (``synth``).
Run from the repository root:

    python tests/golden/make_golden.py           # workloads.json (seconds)
    python tests/golden/make_golden.py --large   # workloads_large.json (tens of minutes)
"""
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
    with open(os.path.join(HERE, "workloads_large.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    if "--large" in sys.argv:
        main_large()
    else:
        main()
