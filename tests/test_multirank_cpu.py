"""The multi-process path on CPU (gloo ranks of torch.distributed):
  * bench.py's timing aggregation: the maximum over ranks and the whole-job throughput;
  * the partition of one batch over ranks (contiguous slices, network replicated, one gather of the
    bounds): each rank bounds its slice with the CPU oracle, and the gathered bounds equal the
    single-process run's, in batch order;
  * a rank that fails on the host surfaces as an error on the other rank's collective instead of a
    hang.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2101_05844_gb300.shard import shard_batch


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    import datetime

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    return dist


def _timing_rank(rank, world, port, out, fail_rank):
    import torch

    import bench
    dist = _init(rank, world, port)
    try:
        if rank == fail_rank:
            raise RuntimeError("injected failure on the host")
        # rank r pretends its step took (10 + r) ms and its end-to-end step (12 + 2 r) ms
        ms, ms_e2e = bench.slowest_rank([10.0 + rank, 12.0 + 2 * rank], dist, torch.device("cpu"))
        out[rank] = (ms, ms_e2e, bench.job_throughput(9 * 2200, world, ms))
        dist.barrier()
    except RuntimeError as e:
        out[rank] = ("error", str(e)[:60])
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _oracle_bounds(prob, lo, hi, C, kw):
    from oracle import active_set as AS
    from oracle import network as nw
    dense = nw.dense_layers(prob["net"])
    out = []
    for s in range(lo.shape[0]):
        P = nw.Problem(prob["net"], lo[s], hi[s], C[s], dense=dense)
        out.append(AS.ActiveSet(P, AS.Options(**kw)).step(kw["bigm_iters"] + kw["as_iters"]).bound())
    return np.array(out)


KW = dict(bigm_iters=6, as_iters=10, omega=4, max_cuts=3)


def _shard_rank(rank, world, port, out):
    import torch

    from paper_2101_05844_gb300 import synth
    from paper_2101_05844_gb300.shard import gather_bounds
    dist = _init(rank, world, port)
    try:
        prob = synth.problem("mlp_4_5_5_1", S=7, seed=3)
        a, b = shard_batch(7, world, rank)
        local = _oracle_bounds(prob, prob["lo"][a:b], prob["hi"][a:b], prob["C"][a:b], KW)
        full = gather_bounds(torch.from_numpy(local), 7, dist)
        out[rank] = full.numpy().tolist()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    import bench
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_timing_rank, args=(world, _free_port(), out, -1), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, ms_e2e, value = res[r]
        assert ms == 11.0 and ms_e2e == 14.0          # the slowest rank's timings on every rank
        assert value == pytest.approx(9 * 2200 * 2 / 0.011)


def test_sharded_oracle_bounds_gather_to_the_single_process_result():
    """7 subproblems over 2 ranks (slices of 4 and 3): the gathered bounds equal, in batch order, the
    bounds of one process bounding the whole batch."""
    from paper_2101_05844_gb300 import synth
    prob = synth.problem("mlp_4_5_5_1", S=7, seed=3)
    ref = _oracle_bounds(prob, prob["lo"], prob["hi"], prob["C"], KW)
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_shard_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        np.testing.assert_array_equal(np.array(res[r]), ref)


def test_shard_slices_cover_the_batch_in_order():
    for S in (0, 1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            slices = [shard_batch(S, world, r) for r in range(world)]
            assert slices[0][0] == 0 and slices[-1][1] == S
            assert all(slices[r][1] == slices[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in slices]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard_batch(4, 2, 2)


def test_a_failing_rank_surfaces_as_an_error_on_the_other():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        try:
            mp.start_processes(_timing_rank, args=(world, _free_port(), out, 1), nprocs=world, start_method="spawn")
        except Exception:
            pass
        res = dict(out)
    assert res[1][0] == "error" and "injected" in res[1][1]
    assert res[0][0] == "error"       # rank 0's collective ends with an error instead of hanging


def test_single_process_needs_no_collective():
    import torch

    import bench
    from paper_2101_05844_gb300.shard import gather_bounds
    assert bench.slowest_rank([3.0, 4.0], None, None) == [3.0, 4.0]
    assert bench.job_throughput(9 * 2200, 1, 1000.0) == 9 * 2200
    t = torch.arange(5, dtype=torch.float64)
    assert gather_bounds(t, 5, None) is t
