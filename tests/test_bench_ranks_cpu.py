"""bench.py with N > 1: one process per GPU, each advancing its own replica
(weak scaling, no data-path collective).  Its rank logic runs here as two
gloo processes on the CPU: the process group forms, the timed region is
bracketed by a barrier, the job's time is the slowest rank's, the whole-job
throughput counts every rank's steps, and the reference arm (the oracle) runs
on rank 0 only while the other ranks return at once."""
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    bench.init_ranks(w, "gloo")
    dist.barrier()
    ms = 100.0 + 50.0 * rank                  # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, w, torch.device("cpu"))
    value = bench.job_throughput(w, 20, slowest)

    class Args:
        steps, warmup, gpus = 2, 3, world
    ref_rc = bench.run_reference(Args()) if rank != 0 else None
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, slowest, value, ref_rc))


def test_two_ranks_time_the_slowest_and_count_every_replica():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=10) for _ in range(2))
    for rank, slowest, value, ref_rc in res:
        assert slowest == 150.0                       # the max over ranks, on every rank
        assert abs(value - 2 * 20 / 0.150) < 1e-9      # both replicas' steps over the slowest time
    assert res[1][3] == 0                              # the reference arm's rank 1 returns without work


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.init_ranks(1, "gloo")
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.job_throughput(1, 10, 500.0) == 20.0
