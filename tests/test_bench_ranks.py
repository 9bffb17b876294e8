"""The multi-rank host logic of bench.py on CPU: two gloo ranks (the same
calls torchrun ranks make on GPUs, with the CPU backend).  Each rank times a
different amount of work; the job time is the slowest rank's, the rate adds
up over ranks (weak scaling), and no two ranks draw the same points."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local, dist = bench._dist()
    assert (r, w, local) == (rank, world, rank) and dist.get_backend() == "gloo"
    elapsed = 1.5 + rank  # rank 1 is the slow one
    job = bench.max_over_ranks(elapsed, dist)
    rate = bench.whole_job_rate(w, 1000, 4, job)
    inst = [bench.rank_instance(i, r, "batched") for i in range(256)]
    ctx = bench.rank_instance(0, r, "bases")
    gathered = [None] * w
    dist.all_gather_object(gathered, (inst, ctx))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, job, rate, gathered))


def test_two_ranks_max_time_and_disjoint_instances():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, job, rate, gathered in res:
        assert job == pytest.approx(2.5)  # the slower rank's time on both
        assert rate == pytest.approx(2 * 1000 * 4 / 2.5)
        (i0, c0), (i1, c1) = gathered
        assert set(i0).isdisjoint(i1) and c0 != c1


def test_single_rank_needs_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.whole_job_rate(1, 10, 2, 4.0) == 5.0
    assert bench.rank_instance(7, 0, "batched") == 7 and bench.rank_instance(0, 0, "vegas") == 0


def test_roofline_operations_are_launch_weighted_for_bases():
    """A BASES step launches ITMX1 refining passes (with the per-bin
    histogram) and ITMX2 frozen-grid passes (without): the operations per
    point are weighted by those launches; a VEGAS step counts every pass in
    full."""
    import bench
    r = bench.Runner.__new__(bench.Runner)
    r.name, r.mode = "dgauss8", "bases"
    r.w = dict(itmx1=5, itmx2=5)
    ops = bench.ALGO_OPS["dgauss8"]
    full, frozen = sum(ops.values()), sum(v for k, v in ops.items() if k != "histogram")
    assert frozen == full - ops["histogram"]
    assert r.ops_per_point() == (5 * full + 5 * frozen) / 10
    r.w = dict(itmx1=3, itmx2=7)
    assert r.ops_per_point() == (3 * full + 7 * frozen) / 10
    r.name, r.mode = "rambo5", "vegas"
    assert r.ops_per_point() == sum(bench.ALGO_OPS["rambo5"].values())
