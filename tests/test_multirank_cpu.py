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


# ----------------------------------------------------------------------------
# Stream placement over devices (gw_partition_streams, host only)
# ----------------------------------------------------------------------------

def _streams(n=64):
    strides = np.array([(128, 256, 512)[i % 3] for i in range(n)], np.int32)
    state = (2 * 21 * 2 * 32768 * 2 + 3 * strides * 4 * 64).astype(np.int64)  # grows with the stride
    return strides, state


def test_partition_balances_load_within_budgets(gpu_free_lib):
    from paper_2108_12430_gb300 import gwstream as G
    strides, state = _streams()
    budgets = np.array([state.sum() // 2 + 10 * state.max()] * 3, np.int64)
    rc, dev, load = G.gw_partition_streams(strides, state, budgets)
    assert rc == G.GW_OK and (dev >= 0).all()
    for d in range(3):
        assert state[dev == d].sum() <= budgets[d]
        np.testing.assert_allclose(load[d], (1.0 / strides[dev == d]).sum())
    # greedy placement in decreasing load: the spread is at most one stream's load
    assert load.max() - load.min() <= 1.0 / strides.min() + 1e-12
    # deterministic: the same arguments give the same placement
    assert (G.gw_partition_streams(strides, state, budgets)[1] == dev).all()


def test_partition_refuses_what_does_not_fit(gpu_free_lib):
    from paper_2108_12430_gb300 import gwstream as G
    strides, state = _streams(9)
    budgets = np.array([state[:4].sum(), -1], np.int64)  # device 1 not available, device 0 holds four streams
    rc, dev, _ = G.gw_partition_streams(strides, state, budgets)
    assert rc == G.GW_EBUDGET
    assert (dev == 0).sum() >= 4 - 1 and (dev == 1).sum() == 0 and (dev == -1).sum() >= 1
    assert state[dev == 0].sum() <= budgets[0]


def test_partition_keeps_streams_whose_device_stays(gpu_free_lib):
    from paper_2108_12430_gb300 import gwstream as G
    strides, state = _streams(30)
    budgets = np.array([state.sum()] * 3, np.int64)
    _, dev, _ = G.gw_partition_streams(strides, state, budgets)
    gone = budgets.copy()
    gone[2] = -1
    rc, dev2, load2 = G.gw_partition_streams(strides, state, gone, current=dev)
    assert rc == G.GW_OK
    assert (dev2[dev != 2] == dev[dev != 2]).all()  # only the lost device's streams move
    assert set(dev2[dev == 2]) <= {0, 1} and load2[2] == 0.0


def _rank_serve(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2108_12430_gb300 import gwstream as G
        strides, state = _streams()
        budgets = np.array([state.sum()] * world, np.int64)  # each rank's device (one per rank)
        rc, dev, _ = G.gw_partition_streams(strides, state, budgets)
        assert rc == G.GW_OK
        mine = [int(i) for i in np.flatnonzero(dev == rank)]  # streams this rank opens and serves
        lists = [None] * world
        dist.all_gather_object(lists, mine)
        placements = [None] * world
        dist.all_gather_object(placements, dev.tolist())
        if rank == 0:
            np.save(os.path.join(out_dir, "served.npy"), np.array(sorted(sum(lists, [])), np.int64))
            np.save(os.path.join(out_dir, "same.npy"), np.array([placements[0] == p for p in placements]))
        dist.barrier()
        if rank == 1:
            return  # rank 1 leaves between steps, with nothing of it in flight
        # rank 0 is told that rank 1 left and places its streams on the ranks that remain
        alive = np.array([r != 1 for r in range(world)])
        rc, dev2, _ = G.gw_partition_streams(strides, state, np.where(alive, budgets, -1), current=dev)
        np.save(os.path.join(out_dir, "rebalance.npy"), np.stack([dev, dev2]))
    finally:
        if rank == 0:
            dist.destroy_process_group()


def test_two_gloo_ranks_share_the_streams_and_rebalance(tmp_path, gpu_free_lib):
    world, port = 2, _free_port()
    mp.start_processes(_rank_serve, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    served = np.load(tmp_path / "served.npy")
    assert (served == np.arange(64)).all()           # every stream served exactly once
    assert np.load(tmp_path / "same.npy").all()      # both ranks computed the same placement
    dev, dev2 = np.load(tmp_path / "rebalance.npy")
    assert (dev2 == 0).all()                         # rank 1's streams moved to rank 0 ...
    assert (dev2[dev == 0] == 0).all()               # ... and rank 0 kept its own
