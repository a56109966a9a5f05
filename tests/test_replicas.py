"""The N-GPU form of bench.py is replicas only: every rank runs its own graph
and batch stream, and the ranks meet only in a barrier and in the reduction
of their times and update counts.  This covers that host logic with two
gloo ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    seconds = 1.0 + r          # rank r "took" 1 + r seconds
    edges = 100.0 * (r + 1)
    t_max = bench.allreduce(w, seconds, "max")
    e_sum = bench.allreduce(w, edges, "sum")
    spec = dict(bench.BENCH["c1"])
    _, keys, _, _, batches = bench.make_batches(spec, 2, r)
    out.put((r, t_max, e_sum, int(keys.size), [b[0].tolist() for b in batches]))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_replicas_reduce_time_and_updates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, e0, m0, b0), (r1, t1, e1, m1, b1) = res
    assert (r0, r1) == (0, 1)
    # max over ranks of the time, sum of the work: value = all updates / slowest rank
    assert t0 == t1 == 2.0 and e0 == e1 == 300.0
    # the same graph on every rank, a different batch stream per rank (weak scaling)
    assert m0 == m1
    assert b0 != b1


@pytest.mark.parametrize("world", [1])
def test_single_process_needs_no_process_group(world):
    sys.path.insert(0, ROOT)
    import bench

    assert bench.allreduce(1, 3.5, "max") == 3.5
    bench.barrier(1)
