"""Write ``workloads.json``: oracle results on the small seeded workloads.

Calls only the CPU oracle (``oracle/``) and the seeded generators (``synth``).
Run from the repository root:  python tests/golden/make_golden.py
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


if __name__ == "__main__":
    main()
