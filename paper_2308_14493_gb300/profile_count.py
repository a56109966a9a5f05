"""Static count of a seeded Chung-Lu graph, repeated, for kernel profiling.

    python -m paper_2308_14493_gb300.profile_count --n 800000 --m 15000000 \\
        --gamma 2.3 --dmax 10000 --reps 2 [--batch 100000 [--batched]] [--local] [--vertex | --edge] [--tuning JSON]

Opens the graph (one static count), then runs ``reps`` more static counts
(or, with ``--batch``, ``reps`` sequential batches of that many updates, 60%
insertions, one ``gc_apply_batch`` call each, or all in one batched call with
``--batched``; with ``--local`` through the edge-local delta; with
``--vertex`` the per-vertex graphlet counts, with ``--edge`` the per-edge
orbit counts) and prints the per-stage device times of each call.  Used as
the command under ncu; it runs the library exactly as a user would.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import gen  # noqa: E402

from . import gc as gcb  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=800000)
    ap.add_argument("--m", type=int, default=15000000)
    ap.add_argument("--gamma", type=float, default=2.3)
    ap.add_argument("--dmax", type=float, default=10000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--autotune", action="store_true", help="pick the bin boundaries first")
    ap.add_argument("--local", action="store_true", help="batches take the edge-local delta")
    ap.add_argument("--batched", action="store_true", help="with --batch: all batches in one batched call")
    ap.add_argument("--vertex", action="store_true", help="per-vertex graphlet counts instead of static counts")
    ap.add_argument("--edge", action="store_true", help="per-edge orbit counts instead of static counts")
    ap.add_argument("--heavy-min", default="",
                    help="with --vertex / --edge: comma-separated local_c4_heavy_min values, each timed in turn")
    ap.add_argument("--chunk-threshold", type=int, default=0,
                    help="wedge bound above which 4-cycle pivots use the chunked shared-memory kernel")
    ap.add_argument("--tuning", default="", help="JSON object of bin boundaries to set after the open "
                                                 "(e.g. '{\"c4_chunk_min\": 262144}'), applied after --autotune")
    a = ap.parse_args()
    keys = gen.chung_lu_graph(a.n, a.m, a.gamma, a.dmax, a.seed)
    rp, col = gen.csr_from_keys(a.n, keys)
    with gcb.Graph(a.n, rp, col, chunk_threshold=a.chunk_threshold,
                   local_max_pairs=(1 << 30) if a.local else 0) as g:
        print(json.dumps({"open": g.stats()["ms_stage"]}), flush=True)
        if a.autotune:
            best, ms = g.autotune(reps=2)
            print(json.dumps({"autotune_ms": ms, "tuning": best}), flush=True)
        if a.tuning:
            g.set_tuning(**json.loads(a.tuning))
            print(json.dumps({"tuning": g.tuning()}), flush=True)
        heavy = [int(x) for x in a.heavy_min.split(",") if x] or [None]
        if a.edge or a.vertex:
            for hm, edge in [(h, ed) for ed in ([False] if a.vertex else []) + ([True] if a.edge else [])
                             for h in heavy]:
                if hm is not None:
                    g.set_tuning(local_c4_heavy_min=hm)
                for _ in range(a.reps):
                    if edge:
                        e, _o = g.edge_orbits()
                        rec = {"edge_orbits_ms": g.stats()["ms_device"], "edges": int(e.shape[0])}
                        del e, _o
                    else:
                        v = g.vertex_counts()
                        rec = {"vertex_counts_ms": g.stats()["ms_device"], "vertices": int(v.shape[0])}
                    rec["local_c4_heavy_min"] = g.tuning()["local_c4_heavy_min"]
                    rec["launches"] = g.stats()["launches"]
                    print(json.dumps(rec), flush=True)
        elif a.batch and a.batched:
            batches = gen.batch_stream(a.n, keys, [a.batch] * a.reps, 0.6, a.seed + 1)
            g.apply_many(batches)
            st = g.stats()
            print(json.dumps({"batches": a.reps, "run_ms": st["ms_device"], "path": st["path"],
                              "launches": st["launches"], "counts": g.counts()}), flush=True)
        elif a.batch:
            for ins, dels in gen.batch_stream(a.n, keys, [a.batch] * a.reps, 0.6, a.seed + 1):
                g.apply(ins, dels)
                st = g.stats()
                print(json.dumps({"batch_ms": st["ms_device"], "stage_ms": st["ms_stage"], "path": st["path"],
                                  "region_vertices": st["region_vertices"], "probes": st["work_triangles"]}),
                      flush=True)
        else:
            for _ in range(a.reps):
                g.count_static()
                st = g.stats()
                print(json.dumps({"static_ms": st["ms_device"], "stage_ms": st["ms_stage"],
                                  "work_triangles": st["work_triangles"], "work_wedges": st["work_wedges"],
                                  "heavy_ms": st["ms_stage"][7], "work_wedges_heavy": st["work_wedges_heavy"],
                                  "l2_red_heavy": st["l2_red_heavy"], "l2_atom_heavy": st["l2_atom_heavy"],
                                  "counts": g.counts()}),
                      flush=True)


if __name__ == "__main__":
    main()
