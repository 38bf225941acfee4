"""The multi-process path of bench.py on CPU: two gloo ranks (torch.distributed), each bounding its
own batch as bench.py's replicas do, aggregate their timings by the maximum over ranks and report
the whole-job throughput; and a rank that fails is reported by the other's collective timing out.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out, fail_rank):
    import datetime

    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure on the host")
        # rank r pretends its step took (10 + r) ms and its end-to-end step (12 + 2 r) ms
        ms, ms_e2e = bench.slowest_rank([10.0 + rank, 12.0 + 2 * rank], dist, torch.device("cpu"))
        out[rank] = (ms, ms_e2e, bench.job_throughput(9, world, ms))
        dist.barrier()
    except RuntimeError as e:
        out[rank] = ("error", str(e)[:60])
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    import bench
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out, -1), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, ms_e2e, value = res[r]
        assert ms == 11.0 and ms_e2e == 14.0          # the slowest rank's timings on every rank
        assert value == pytest.approx(9 * bench.iterations_per_step() * 2 / 0.011)


def test_a_failing_rank_surfaces_as_an_error_on_the_other():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        try:
            mp.start_processes(_rank_main, args=(world, _free_port(), out, 1), nprocs=world, start_method="spawn")
        except Exception:
            pass
        res = dict(out)
    assert res[1][0] == "error" and "injected" in res[1][1]
    assert res[0][0] == "error"       # rank 0's collective ends with an error instead of hanging


def test_single_process_needs_no_collective():
    import bench
    assert bench.slowest_rank([3.0, 4.0], None, None) == [3.0, 4.0]
    assert bench.job_throughput(9, 1, 1000.0) == 9 * bench.iterations_per_step()
