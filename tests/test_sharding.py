"""Sharding trajectories over ranks (gloo, world size 2, CPU).

Each rank runs the oracle on its contiguous block of global trajectory ids;
the merged moments must equal those of one process running every trajectory,
and every per-trajectory result must be identical (counter-based RNG keyed by
the global id).
"""
import os
import socket

import numpy as np
import torch.multiprocessing as tmp

from paper_2501_17913_gb300.shard import PeerFailure, job_rate, merge_ensemble, report_alive, shard_range, wait_peers


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _job(traj):
    from oracle_jobs import run_traj
    return run_traj(("config_small_fp64", {"n_traj": 10}, traj, {"n_steps": 8}))[0]


def _rank_main(rank, world, port, n_total, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = shard_range(n_total, rank, world)
    vals = np.array([_job(t) for t in range(first, first + count)])
    np.save(os.path.join(outdir, "rank%d.npy" % rank), vals)
    mean, sem = merge_ensemble(vals)
    if rank == 0:
        np.save(os.path.join(outdir, "merged.npy"), np.stack([mean, sem]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_ids_once():
    for n in (1, 7, 10, 1024):
        for world in (1, 2, 3, 8):
            ids = []
            for r in range(world):
                f, c = shard_range(n, r, world)
                ids += list(range(f, f + c))
            assert ids == list(range(n))


def test_two_rank_merge_equals_single_process(tmp_path):
    n_total, world = 10, 2
    port = _free_port()
    tmp.start_processes(_rank_main, args=(world, port, n_total, str(tmp_path)), nprocs=world, join=True,
                        start_method="spawn")
    parts = [np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world)]
    allv = np.concatenate(parts)
    single = np.array([_job(t) for t in range(n_total)])
    assert np.array_equal(allv, single)
    merged = np.load(tmp_path / "merged.npy")
    assert np.allclose(merged[0], single.mean(axis=0), atol=1e-15)
    assert np.allclose(merged[1], single.std(axis=0, ddof=1) / np.sqrt(n_total), atol=1e-15)


def _rate_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, ms = (100.0, 1000.0) if rank == 0 else (300.0, 2000.0)
    value, t_max = job_rate(units, ms)
    np.save(os.path.join(outdir, "rate%d.npy" % rank), np.array([value, t_max]))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_is_all_units_over_the_slowest_rank(tmp_path):
    """The benchmark's whole-job value under torchrun: sum of units / max of times, on every rank."""
    world = 2
    tmp.start_processes(_rate_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                        start_method="spawn")
    for r in range(world):
        value, t_max = np.load(tmp_path / ("rate%d.npy" % r))
        assert t_max == 2000.0 and value == 400.0 / 2.0
    assert job_rate(50.0, 500.0) == (100.0, 500.0)      # no process group: the local rate


def _heartbeat_main(rank, world, port, outdir):
    from datetime import timedelta

    import torch.distributed as dist
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=timedelta(seconds=30))
    report_alive(store, rank, "step0")
    wait_peers(store, world, "step0", 20.0)          # every rank finishes step 0
    if rank == 1:
        return                                        # rank 1 leaves between steps (a failed rank)
    report_alive(store, rank, "step1")
    try:
        wait_peers(store, world, "step1", 2.0)
        result = "no failure seen"
    except PeerFailure as e:
        result = str(e)
    with open(os.path.join(outdir, "rank0.txt"), "w") as f:
        f.write(result)


def test_a_rank_that_leaves_is_noticed_on_the_host(tmp_path):
    """Failure detection without any device fault: the surviving rank learns from the store, before
    its next launch, that rank 1 is gone."""
    tmp.start_processes(_heartbeat_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                        start_method="spawn")
    msg = open(tmp_path / "rank0.txt").read()
    assert "ranks [1]" in msg and "step1" in msg
