"""The bench's multi-rank logic on CPU: two gloo ranks (world size 2).

Under torchrun every rank runs an independent replica of the streaming path
on its own GPU (streams are independent, so there is no data-path
collective); the ranks meet only at barriers and in the max-reduction of the
timed interval, and rank 0 reports the whole-job rate.  This test runs that
host logic with the gloo backend and checks the slowest rank's time, the
whole-job rate and the per-rank input seeds.
"""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.rank_env()
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = 100.0 + 25.0 * rank          # rank 1 is the slowest replica
        t = bench.slowest(dist, world, local_ms, "cpu")
        rate = bench.job_rate(64 * 10, world, t / 1e3)
        wit, _ = bench.make_stream_inputs(4096, seed=1234 + rank)
        dist.barrier()
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([t, rate, wit[0, :8].sum()]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    r0, r1 = np.load(tmp_path / "rank0.npy"), np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 125.0                      # both ranks see the max
    assert abs(r0[1] - 64 * 10 * 2 / 0.125) < 1e-9      # units of all ranks / slowest time
    assert r0[2] != r1[2]                               # each replica streams its own inputs


def test_single_rank_needs_no_collective():
    import bench
    assert bench.slowest(None, 1, 3.5, "cpu") == 3.5
    assert bench.job_rate(640, 1, 2.0) == 320.0
