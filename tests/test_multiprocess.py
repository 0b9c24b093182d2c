"""The multi-GPU path is replicas only: each rank tracks its own frames and the
job's time is the maximum over ranks.  These world-size-2 gloo runs on the CPU
cover the host logic the benchmark uses under torchrun: distinct shards per
rank, the max-over-ranks time and the summed units, and that a frame's result
does not depend on which rank processed it."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle as orc
        from paper_2509_10757_gb300 import scenes
        seed = bench.shard_seed(0, rank)
        frames = scenes.pinhole_batch(seed=seed, n_frames=2, nl_range=(200, 300), m_range=(200, 300))
        kp, mpu = bench.units_of(frames)
        t_local = 1.0 + rank                      # pretend rank r took 1 + r seconds
        t_job = bench.max_over_ranks(t_local, world)
        units = bench.sum_over_ranks(float(kp + mpu), world)
        st, se = orc.track_frame(dict(scenes.DEFAULT_PARAMS), frames[0])
        q.put((rank, seed, t_job, units, kp + mpu, st["u_right"].tobytes(), se["mp_kp"].tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    seeds = [r[1] for r in res]
    assert len(set(seeds)) == world, "every rank gets its own frames"
    assert all(r[2] == 2.0 for r in res), "job time is the max over ranks"
    total = sum(r[4] for r in res)
    assert all(r[3] == total for r in res), "units are summed over ranks"
    # a frame tracked on rank 1 gives the same result when tracked here
    import oracle as orc
    import bench
    from paper_2509_10757_gb300 import scenes
    fr = scenes.pinhole_batch(seed=bench.shard_seed(0, 1), n_frames=2, nl_range=(200, 300),
                              m_range=(200, 300))[0]
    st, se = orc.track_frame(dict(scenes.DEFAULT_PARAMS), fr)
    assert st["u_right"].tobytes() == res[1][5]
    assert se["mp_kp"].tobytes() == res[1][6]
