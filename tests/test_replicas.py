"""Multi-rank host logic (replicas, no data-path collective) on CPU with gloo, world size 2."""
import os
import socket

import pytest

from paper_2005_11976_gb300 import replicas


def test_shard_partitions_every_scan_once():
    for n in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_whole_job_rate():
    assert replicas.whole_job_rate(20.0, 4, 2.0) == pytest.approx(40.0)
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1.0, 1, 0.0)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, local = replicas.dist_env()
    assert (r, w, local) == (rank, world, rank)
    replicas.init("gloo")
    replicas.barrier()
    mine = replicas.shard(10, r, w)
    t_max = replicas.max_over_ranks(times[r])
    replicas.barrier()
    out.put((r, mine, t_max, replicas.whole_job_rate(len(mine), w, t_max)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_meet_only_in_the_timing_reduction():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.5, 2.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [[0, 2, 4, 6, 8], [1, 3, 5, 7, 9]]
    assert all(r[2] == pytest.approx(2.5) for r in res)   # the slowest rank's time
    assert all(r[3] == pytest.approx(5 * 2 / 2.5) for r in res)


def _batch_rank(rank, world, port, out):
    # a batch of 7 scan descriptions sharded over the ranks; each rank "reconstructs" its
    # scans (a deterministic function of the scan's seeded inputs stands in for the GPU
    # solve) and rank 0 gathers the per-scan results in the batch's order
    import numpy as np
    from paper_2005_11976_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    replicas.init("gloo")
    scans = synth.batched_scans(7)
    mine = replicas.shard(len(scans), rank, world)
    vals = [(i, scans[i].n_proj, float(np.round(scans[i].tx, 12))) for i in mine]
    got = replicas.gather_ordered(vals, len(scans), rank, world)
    out.put((rank, got))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_shard_a_batch_and_gather_results_in_order():
    import torch.multiprocessing as mp
    from paper_2005_11976_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    scans = synth.batched_scans(7)
    assert res[1] is None
    assert res[0] == [(i, s.n_proj, float(round(s.tx, 12))) for i, s in enumerate(scans)]
    # one process: the list comes back as it is
    assert replicas.gather_ordered([1, 2], 2, 0, 1) == [1, 2]
    with pytest.raises(ValueError):
        replicas.gather_ordered([1], 4, 0, 2)

