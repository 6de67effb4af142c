"""The benchmark's multi-rank bookkeeping on CPU (gloo, two ranks).

Under torchrun every rank runs its own replica of the workload (weak scaling,
no collective on the data path); the ranks agree on the slowest rank's time
and rank 0 reports the whole-job grind time over the cells of all ranks.  The
GPU work itself needs no exchange, so this is the whole of the N > 1 path."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    t = bench.max_over_ranks(0.25 + 0.5 * rank, world)      # ranks took 0.25 s and 0.75 s
    g = bench.aggregate_grind(t, steps=10, ncell=1000, neq=7, world=world)
    out.put((r, w, local, t, g))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time_and_aggregate_the_cells():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, t, g) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert t == 0.75
        # 0.75 s over 2 replicas x 10 steps x 3 RHS x 1000 cells x 7 eq
        assert g == pytest.approx(0.75e9 / (10 * 3 * 1000 * 7 * 2), rel=1e-15)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.aggregate_grind(2.0, 4, 100, 5, 1) == pytest.approx(2e9 / (4 * 3 * 100 * 5))
